// g6gb_kernels.cu -- sm_103a kernels of the direct-summation hot path
// (Gaburov, Harfst & Portegies Zwart, arXiv:0902.4463):
//
//   K0 k_scatter      j-memory update from staged records      (Sect. 2.1)
//   K1 k_predict_*    j-particle prediction, Eq. 1 and Eq. 2   (Sect. 2.2)
//   K2 k_force_ds     FP32 pair forces with double-single separations,
//                     Eq. 3, nearest neighbour, neighbour lists (Sect. 2.3, 2.5, 4)
//   K2d k_force_64    the same in FP64
//   K3 k_reduce       reduction of the partial forces          (Sect. 2.3)
//                     (compensated FP32 for the DS path, FP64 for the FP64 path)
//
// Work partition of K2/K2d.  The paper spreads the j-particles over the
// multiprocessors, gives every block all i-particles, cuts i into serial
// segments when there are too many, and splits j again inside a block when
// the active block is small (Sect. 2.3, Figs. accGPU, accMP, accMP1).  Here
// the (i-tile, j-tile) pairs form one work line that is cut into `grid`
// equal contiguous ranges, one per resident CTA, so every SM gets the same
// number of pair tiles whatever m and n are.  A CTA that crosses an i-tile
// boundary writes one partial per i-tile it touched; K3 sums the partials of
// each i in FP64.  Inside a CTA, TJ thread groups split each j-tile when m is
// small (the split-j of Fig. accMP1).
//
// j-tiles are staged in shared memory by bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier) issued by one thread, in a
// NSTAGE-deep ring, so the loads of later tiles overlap the pair loop.  Every
// mbarrier wait is bounded; on expiry the kernel records G6_ETIMEDOUT in the
// error word, waits (bounded) for its own copies in flight and returns.
#include "g6gb_device.cuh"

#include <climits>
#include <cmath>
#include <type_traits>

namespace g6 {

namespace {

constexpr int NSTAGE = 3;
constexpr int FP_NSTAGE = 2;        // raw-tile stages of the fused-prediction kernels

}  // namespace

// ----------------------------------------------------------------- K0 ---

__global__ void k_init_store(JStore js)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < js.cap;
         k += gridDim.x * blockDim.x) {
        js.x0[k] = FAR;
        js.x0[js.cap + k] = FAR;
        js.x0[2 * js.cap + k] = FAR;
        js_xds(js, k) = make_float4((float)FAR, (float)FAR, (float)FAR, 0.f);
        js_xds2(js, k) = make_float2(0.f, 0.f);
        js_t0(js, k) = 0.0;
        js_v0m(js, k) = make_float4(0.f, 0.f, 0.f, 0.f);
        js_a2f(js, k) = make_float4(0.f, 0.f, 0.f, 0.f);
        js_j6f(js, k) = make_float4(0.f, 0.f, 0.f, 0.f);
        js.v64[k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        js.a264[k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        js.j664[k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        js.idx[k] = -1;
        js_idx(js, k) = -1;
    }
}


// K0: one thread per record; addresses within one launch are distinct (the
// host staging keeps one record per address).
__global__ void k_scatter(const g6x_jrec *__restrict__ rec, int n, JStore js)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n)
        store_record(rec[k], js);
}

// Tuning input: i-records built from the first m j-slots of j-memory.
__global__ void k_irec_from_store(JStore js, g6x_irec *out, int m)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m || k >= js.cap)
        return;
    g6x_irec r;
    r.x[0] = js.x0[k];
    r.x[1] = js.x0[js.cap + k];
    r.x[2] = js.x0[2 * js.cap + k];
    double4_32a v = js.v64[k];
    r.v[0] = v.x;
    r.v[1] = v.y;
    r.v[2] = v.z;
    r.h2 = 0.0;
    r.index = js.idx[k];
    r.pad = 0;
    out[k] = r;
}

// ----------------------------------------------------------------- K1 ---


// Records one tile's range of particle indices (empty slots excluded);
// called by all JT threads of the CTA with their own slot's index.  The
// per-warp ranges go to the half `par` of the double-buffered s_lo / s_hi,
// so consecutive tiles need only the one barrier here: the next tile writes
// the other half, and the tile after that passes this tile's barrier after
// thread 0 has read its half.
__device__ __forceinline__ void tile_index_range(int (*s_lo)[JT / 32], int (*s_hi)[JT / 32],
                                                 int par, int id, bool valid, int2 *out)
{
    int lo_id = valid ? id : INT_MAX, hi_id = valid ? id : -1;
    lo_id = __reduce_min_sync(0xffffffffu, lo_id);
    hi_id = __reduce_max_sync(0xffffffffu, hi_id);
    if ((threadIdx.x & 31) == 0) {
        s_lo[par][threadIdx.x >> 5] = lo_id;
        s_hi[par][threadIdx.x >> 5] = hi_id;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < JT / 32; ++w) {
            lo_id = min(lo_id, s_lo[par][w]);
            hi_id = max(hi_id, s_hi[par][w]);
        }
        *out = make_int2(lo_id, hi_id);
    }
}

// Eq. 1 and Eq. 2 for one j-slot k < nj in the paper's DS + SP form
// (predict_ds_vals), written to the tiled DS layout.
__device__ __forceinline__ void predict_slot_ds(const JStore &js, int k, double t, float *o,
                                                int id)
{
    predict_ds_vals((float)(t - js_t0(js, k)), js_xds(js, k), js_xds2(js, k), js_v0m(js, k),
                    js_a2f(js, k), js_j6f(js, k), id, o);
}

// The same with the DS position formed through FP64: the FP32 increment is
// added to the FP64 x0 and the sum split into hi = rn(x), lo = rn(x - hi).
__device__ __forceinline__ void predict_slot_ds_x64(const JStore &js, int k, double t, float *o,
                                                    int id)
{
    const double dt = t - js_t0(js, k);
    const float h = (float)dt;
    const float4 v = js_v0m(js, k), a = js_a2f(js, k), j = js_j6f(js, k);
    const double px = js.x0[k] + (double)(h * fmaf(h, fmaf(h, j.x, a.x), v.x));
    const double py = js.x0[js.cap + k] + (double)(h * fmaf(h, fmaf(h, j.y, a.y), v.y));
    const double pz = js.x0[2 * js.cap + k] + (double)(h * fmaf(h, fmaf(h, j.z, a.z), v.z));
    const float hx = __double2float_rn(px), hy = __double2float_rn(py),
                hz = __double2float_rn(pz);
    const float h3 = 3.0f * h;
    o[W_XH * JT] = hx;
    o[W_YH * JT] = hy;
    o[W_ZH * JT] = hz;
    o[W_M * JT] = v.w;
    o[W_XL * JT] = __double2float_rn(px - (double)hx);
    o[W_YL * JT] = __double2float_rn(py - (double)hy);
    o[W_ZL * JT] = __double2float_rn(pz - (double)hz);
    o[W_VX * JT] = fmaf(h, fmaf(h3, j.x, 2.0f * a.x), v.x);
    o[W_VY * JT] = fmaf(h, fmaf(h3, j.y, 2.0f * a.y), v.y);
    o[W_VZ * JT] = fmaf(h, fmaf(h3, j.z, 2.0f * a.z), v.z);
    o[W_ID * JT] = __int_as_float(id);
}

// Eq. 1 and Eq. 2 entirely in FP64, for the FP64 force kernel.
__device__ __forceinline__ void predict_slot_64(const JStore &js, Pred &p, int k, int nj, double t)
{
    if (k < nj) {
        const double h = t - js_t0(js, k);
        const double4_32a v = js.v64[k], a = js.a264[k], j = js.j664[k];
        const double px = js.x0[k] + h * fma(h, fma(h, j.x, a.x), v.x);
        const double py = js.x0[js.cap + k] + h * fma(h, fma(h, j.y, a.y), v.y);
        const double pz = js.x0[2 * js.cap + k] + h * fma(h, fma(h, j.z, a.z), v.z);
        const double h3 = 3.0 * h;
        const double vx = fma(h, fma(h3, j.x, 2.0 * a.x), v.x);
        const double vy = fma(h, fma(h3, j.y, 2.0 * a.y), v.y);
        const double vz = fma(h, fma(h3, j.z, 2.0 * a.z), v.z);
        p.p64[k] = make_double4_32a(px, py, pz, v.w);
        p.v64[k] = make_double4_32a(vx, vy, vz, (double)js.idx[k]);
    } else {
        p.p64[k] = make_double4_32a(FAR, FAR, FAR, 0.0);
        p.v64[k] = make_double4_32a(0.0, 0.0, 0.0, -1.0);
    }
}

// K1: one CTA of JT threads per tile of j-slots (grid-stride over tiles).
// With UPD, the CTA first stores the staged j-records that fall in its tile
// (rec sorted by tile, tile t's records at [toff[t], toff[t+1])) -- the K0
// update fused into the same launch -- then predicts the tile.  Tiles at or
// beyond the predicted range only take their updates.  The DS kinds also
// record each tile's range of particle indices.
template <int KIND, bool UPD>
__global__ void __launch_bounds__(JT) k_predict(JStore js, Pred p, int nj, int nj_pad,
                                                double t, const g6x_jrec *__restrict__ rec,
                                                const int *__restrict__ toff, int ntiles_all)
{
    grid_dep_launch();              // the force kernel may be scheduled behind this one
    __shared__ int s_lo[2][JT / 32], s_hi[2][JT / 32];
    const int ntiles_pred = nj_pad / JT;
    const int ntiles = UPD ? ntiles_all : ntiles_pred;
    int par = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if constexpr (UPD) {
            for (int r = toff[tile] + threadIdx.x; r < toff[tile + 1]; r += JT)
                store_record(rec[r], js);
            __syncthreads();
        }
        if (tile >= ntiles_pred)
            continue;
        const int k = tile * JT + threadIdx.x;
        if constexpr (KIND == PRED_FP64) {
            predict_slot_64(js, p, k, nj, t);
        } else {
            float *o = p.pt + (size_t)tile * (JW * JT) + threadIdx.x;
            const int id = k < nj ? js_idx(js, k) : -1;
            tile_index_range(s_lo, s_hi, par, id, k < nj && id >= 0, &p.trange[tile]);
            par ^= 1;
            if (k >= nj)
                far_slot_ds(o);
            else if constexpr (KIND == PRED_DS)
                predict_slot_ds(js, k, t, o, id);
            else
                predict_slot_ds_x64(js, k, t, o, id);
        }
    }
}

// K1 for a batch of clusters (tables described with BatchPredTables).
template <int KIND>
__global__ void __launch_bounds__(JT) k_predict_batch(JStore js, Pred p, BatchPredTables bp,
                                                      const g6x_jrec *__restrict__ rec,
                                                      const int *__restrict__ toff, int tile0,
                                                      int ntiles)
{
    __shared__ int s_lo[2][JT / 32], s_hi[2][JT / 32];
    int par = 0;
    for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
        const int tile = tile0 + tt;
        if (rec && toff) {
            for (int r = toff[tile] + threadIdx.x; r < toff[tile + 1]; r += JT)
                store_record(rec[r], js);
            __syncthreads();
        }
        const int k = bp.tile_cluster[tile];
        if (bp.cl_ni[k] <= 0)
            continue;                                  // cluster idle this step
        const int local = (tile - bp.cl_jtile[k]) * JT + threadIdx.x;
        const int slot = tile * JT + threadIdx.x;
        const bool valid = local < bp.cl_nj[k];
        const double t = bp.cl_t[k];
        if constexpr (KIND == PRED_FP64) {
            predict_slot_64(js, p, slot, valid ? slot + 1 : slot, t);
        } else {
            float *o = p.pt + (size_t)tile * (JW * JT) + threadIdx.x;
            const int id = valid ? js_idx(js, slot) : -1;
            tile_index_range(s_lo, s_hi, par, id, valid && id >= 0, &p.trange[tile]);
            par ^= 1;
            if (!valid)
                far_slot_ds(o);
            else if constexpr (KIND == PRED_DS)
                predict_slot_ds(js, slot, t, o, id);
            else
                predict_slot_ds_x64(js, slot, t, o, id);
        }
    }
}

// Separation of two DS positions by the full DS subtraction (the accuracy
// ablation of Sect. 2.3): TwoSum of the high parts, the low parts added to
// its error, one final rounding -- nine FP32 operations against the three
// of Eq. 3.  nh, nl are the negated high and low parts of x_i.
__device__ __forceinline__ float ds_sep1(float h, float l, float nh, float nl)
{
    const float s = __fadd_rn(h, nh);
    const float bb = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(nh, bb));
    return __fadd_rn(s, __fadd_rn(e, __fadd_rn(l, nl)));
}

__device__ __forceinline__ float2 ds_sep2(float2 h, float2 l, float2 nh, float2 nl)
{
    const float2 s = __fadd2_rn(h, nh);
    const float2 bb = __fadd2_rn(s, make_float2(-h.x, -h.y));
    const float2 sb = __fadd2_rn(s, make_float2(-bb.x, -bb.y));
    const float2 e = __fadd2_rn(__fadd2_rn(h, make_float2(-sb.x, -sb.y)),
                                __fadd2_rn(nh, make_float2(-bb.x, -bb.y)));
    return __fadd2_rn(s, __fadd2_rn(e, __fadd2_rn(l, nl)));
}

// ----------------------------------------------------------------- K2 ---


// Pair forces in FP32 with the DS separation of Eq. 3 (Sect. 2.3).  Per pair:
//   dx   = (xj_hi - xi_hi) + (xj_lo - xi_lo)                       Eq. 3
//   r2   = |dx|^2 + eps2, or +inf for the i-particle's own j (index match)
//   1/r  = rsqrt(r2), 1/r^2 = rcp(r2)    (+inf -> 0: the pair adds nothing)
//          (the reciprocal rounds once where 1/r * 1/r compounds the error
//          of the approximate rsqrt, and takes one FMA-pipe operation off)
//   acc  += m r^-3 dx
//   jerk += m r^-3 (dv - 3 (dx.dv) r^-2 dx)
//   pot  += m r^-1                      (negated in K3)
// The softened r2 is also the key of the nearest neighbour and of the lists
// (against h2 + eps2); the partial records carry the neighbour's distance
// with eps2 taken off again.  32 FP32 lane operations per pair.
// Each thread holds NI i-particles and walks its share of every j-tile two
// j-particles at a time: the pair of j values of one component is one float2
// and the arithmetic uses the packed FP32x2 instructions of sm_100+, which
// issue two lanes of FP32 work per instruction.  Subtractions are additions
// of the pre-negated i values (exact).
//
// The per-pair self test is needed only on j-tiles whose index range holds
// one of the warp's i-particles; other tiles take the same loop without it.
// The nearest neighbour is tracked lazily: a running minimum of the key per
// tile and the tile that lowered it; when a segment ends, that one tile is
// scanned again with the same arithmetic to find the first j that attains
// the minimum (ties to the lower j-slot).  Lists (Sect. 4) use the same
// minimum: the loop keeps it per chunk of j-pairs, and only a chunk whose
// minimum is below h2 + eps2 is scanned again, from the staged tile, for
// its members, so the pair loop is the same with and without lists.  With
// TJ j-groups each group keeps its own ascending run of members, and the
// runs are merged when a segment ends.
//
// Sums run in FP32 over one flush interval (>= 512 j per thread) and are
// then folded into compensated (TwoSum) FP32 pairs kept in shared memory, so
// rounding does not grow with n; the pairs are combined in FP64 when
// partials are written.
template <int TI, int TJ, int NI, bool LIST, int MINB = 1, int UNR = 2, bool BATCH = false,
          bool FP = false, bool DSS = false>
__global__ void __launch_bounds__(TI * TJ, MINB) k_force_ds(const ForceArgs a)
{
    static_assert(!(LIST && BATCH), "batches carry no neighbour lists");
    static_assert(!(FP && (LIST || BATCH)), "fused prediction: single context, no lists");
    constexpr int NT = TI * TJ;
    constexpr int ITILE = TI * NI;
    constexpr int PPT = JT / 2 / TJ;                  // j-pairs per thread per tile
    constexpr int FLUSH = (256 + PPT - 1) / PPT;      // tiles between flushes (>= 512 j)
    // The split-j shapes (small m) also note which chunk of CHP j-pairs
    // lowered a tile's minimum, so the rescan at the end of a segment reads
    // one chunk of the winning tile, not the thread's whole share of it.
    // Lists test each chunk's minimum against the radius: whole j-tiles per
    // thread take chunks of 16 j-pairs (4 cost the loop 8 %).
    constexpr bool NNC = TJ > 1;
    constexpr int CHW = NNC ? 4 : 16;
    constexpr int CHP = PPT < CHW ? PPT : CHW;
    static_assert(PPT % CHP == 0, "whole chunks per tile");
    constexpr unsigned TILE_BYTES = JW * JT * sizeof(float);
    // FP: a stage holds one tile of the raw j-store arrays (RAW_* offsets),
    // predicted by the CTA into pbuf before the pair loop
    constexpr unsigned STAGE_BYTES = FP ? RAW_TILE_BYTES : TILE_BYTES;
    constexpr int NS = FP ? FP_NSTAGE : NSTAGE;         // stages in the ring
    static_assert(JT % (2 * TJ) == 0, "j-tile must split into j-pairs evenly");
    // nothing is read before the predecessor (prediction, or an earlier
    // reduction of the same partial buffers) has completed
    grid_dep_wait();
    grid_dep_launch();

    extern __shared__ __align__(128) unsigned char dyn_smem[];
    float *stage_buf = reinterpret_cast<float *>(dyn_smem);
    float *pbuf = reinterpret_cast<float *>(dyn_smem + NS * STAGE_BYTES);    // FP only
    float2 *comp = reinterpret_cast<float2 *>(dyn_smem + NS * STAGE_BYTES
                                              + (FP ? TILE_BYTES : 0));         // [NI][7][NT]
    __shared__ int s_wlo[FP ? NT / 32 : 1], s_whi[FP ? NT / 32 : 1];
    __shared__ __align__(8) uint64_t bar[NS];
    __shared__ int s_abort;
    __shared__ float s_nnr[TJ > 1 ? NI * NT : 1];
    __shared__ int s_nnj[TJ > 1 ? NI * NT : 1];
    // split-j lists: each thread's run of entries (its count, then the head
    // of the run during the merge at the end of a segment)
    constexpr bool LRUN = LIST && TJ > 1;
    __shared__ int s_nbn[LRUN ? NI * NT : 1];
    __shared__ int s_nbh[LRUN ? NI * NT : 1];
    __shared__ float s_ibuf[TJ > 1 ? 11 * ITILE : 1];

    const int tid = threadIdx.x;
    const int ti = tid % TI, tj = tid / TI;
    const long long G = gridDim.x, c = blockIdx.x;
    // Work geometry: global i-tile g of a work position, its work range, its
    // j-tile for a position, and where its i-records and results live.
    long long W;
    int ngt = 0;
    const BatchGT *gt = nullptr;
    if constexpr (BATCH) {
        W = a.bt.hdr[0];
        ngt = (int)a.bt.hdr[1];
        gt = a.bt.gt + a.bt.hdr[2];
    } else {
        W = a.W;
    }
    auto g_start = [&](int g) -> long long {
        if constexpr (BATCH)
            return gt[g].start;
        else
            return (long long)g * a.J;
    };
    auto g_of = [&](long long p) -> int {       // largest g with g_start(g) <= p
        if constexpr (BATCH) {
            int lo = 0, hi = ngt - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (gt[mid].start <= p)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            return lo;
        } else {
            return (int)(p / a.J);
        }
    };
    auto jt_of = [&](long long p, int g) -> int {
        if constexpr (BATCH)
            return a.bt.cl_jtile[gt[g].cluster] + (int)(p - gt[g].start);
        else
            return (int)(p - (long long)g * a.J);
    };
    // record index of slot il of i-tile g, or -1 past the active block
    auto i_index = [&](int g, int il) -> long long {
        if constexpr (BATCH) {
            const int k = gt[g].cluster;
            const int li = gt[g].itile * ITILE + il;
            return li < a.bt.cl_ni[k] ? (long long)a.bt.cl_ioff[k] + li : -1;
        } else {
            const long long gi = (long long)g * ITILE + il;
            return gi < a.ni ? gi : -1;
        }
    };

    const long long wb = work_begin(c, W, G), we = work_begin(c + 1, W, G);
    const int ntile = (int)(we - wb);
    if (ntile <= 0)
        return;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s)
            mbar_init(&bar[s], 1);
        fence_barrier_init();
        s_abort = 0;
    }
    __syncthreads();

    int issue_g = g_of(wb);                     // used by thread 0 only
    auto issue = [&](int q) {
        const long long p = wb + q;
        while (g_start(issue_g + 1) <= p)
            ++issue_g;
        const int jt = jt_of(p, issue_g);
        int s = q % NS;
        if constexpr (FP) {
            unsigned char *d = dyn_smem + (size_t)s * RAW_TILE_BYTES;
            mbar_expect_tx(&bar[s], RAW_TILE_BYTES);
            bulk_g2s(d, raw_tile(a.js, jt), RAW_TILE_BYTES, &bar[s]);
        } else {
            mbar_expect_tx(&bar[s], TILE_BYTES);
            bulk_g2s(stage_buf + (size_t)s * JW * JT, a.pt + (size_t)jt * JW * JT, TILE_BYTES,
                     &bar[s]);
        }
    };

    // FP: Eq. 1 and Eq. 2 for the staged raw tile jt (stage s) into pbuf, with
    // the arithmetic of K1 (bit-identical tiles); each warp's range of
    // particle indices goes to s_wlo/s_whi.
    auto predict_tile = [&](int s, int jt) {
        const unsigned char *d = dyn_smem + (size_t)s * RAW_TILE_BYTES;
        const double *T0 = reinterpret_cast<const double *>(d + RAW_T0);
        const float4 *V = reinterpret_cast<const float4 *>(d + RAW_V);
        const float4 *A = reinterpret_cast<const float4 *>(d + RAW_A);
        const float4 *J = reinterpret_cast<const float4 *>(d + RAW_J);
        const float4 *XA = reinterpret_cast<const float4 *>(d + RAW_XA);
        const float2 *XB = reinterpret_cast<const float2 *>(d + RAW_XB);
        const int *ID = reinterpret_cast<const int *>(d + RAW_ID);
        int lo = INT_MAX, hi = -1;
        for (int jj = tid; jj < JT; jj += NT) {
            float *o = pbuf + jj;
            if (jt * JT + jj < a.nj) {
                const int id = ID[jj];
                predict_ds_vals((float)(a.t_pred - T0[jj]), XA[jj], XB[jj], V[jj], A[jj], J[jj],
                                id, o);
                if (id >= 0) {
                    lo = min(lo, id);
                    hi = max(hi, id);
                }
            } else {
                far_slot_ds(o);
            }
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if ((tid & 31) == 0) {
            s_wlo[tid >> 5] = lo;
            s_whi[tid >> 5] = hi;
        }
    };
    if constexpr (FP) {
        // staged j-records of this CTA's tiles (one i-tile: no other CTA
        // reads these tiles), stored before the bulk copies read them
        if (a.rec) {
            for (int q = 0; q < ntile; ++q) {
                const int jt = (int)(wb + q);
                for (int r = a.toff[jt] + tid; r < a.toff[jt + 1]; r += NT)
                    store_record(a.rec[r], a.js);
            }
            fence_proxy_async_global();
            __syncthreads();
        }
    }
    if (tid == 0)
        for (int q = 0; q < NS && q < ntile; ++q)
            issue(q);

    float2 eps2 = make_float2((float)a.eps2, (float)a.eps2);
    const float2 m3 = make_float2(-3.0f, -3.0f);
    const float INF = __int_as_float(0x7f800000);
    float2 nxh[NI][3], nxl[NI][3], nv[NI][3];
    float h2[NI];
    int iid[NI];
    float2 ta[NI][7];
    float tmin[NI], nnr[NI];
    int nnt[NI], nbn[NI];
    int tchk[NI], nnc[NI];              // NNC: chunk of the tile / of tile nnt
    int cur_t = -1;
    int since_flush = 0;

    auto cslot = [&](int k, int q) -> float2 & { return comp[(k * 7 + q) * NT + tid]; };

    auto flush = [&]() {
#pragma unroll
        for (int k = 0; k < NI; ++k)
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                float2 hl = cslot(k, q);
                float s, e;
                two_sum(hl.x, ta[k][q].x, s, e);
                hl.y = __fadd_rn(hl.y, e);
                two_sum(s, ta[k][q].y, hl.x, e);
                hl.y = __fadd_rn(hl.y, e);
                cslot(k, q) = hl;
                ta[k][q] = make_float2(0.f, 0.f);
            }
    };

    // The DS split of the i-positions (FP64, slow on GB300) is done once per
    // i-particle: with TJ > 1 by the thread whose j-group is 0, shared with the
    // other groups through shared memory.
    auto load_i = [&](int t) {
        if constexpr (BATCH) {
            const float e = (float)a.bt.cl_eps2[gt[t].cluster];
            eps2 = make_float2(e, e);
        }
        if constexpr (TJ > 1) {
            for (int il = tid; il < ITILE; il += NT) {
                const long long gi = i_index(t, il);
                float w[11];
                if (gi >= 0) {
                    const g6x_irec &r = a.irec[gi];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const double x = r.x[d];
                        const float hi = __double2float_rn(x);
                        w[d] = hi;
                        w[3 + d] = __double2float_rn(x - (double)hi);
                        w[6 + d] = (float)r.v[d];
                    }
                    w[9] = (float)(r.h2 + (double)eps2.x);
                    w[10] = __int_as_float(r.index);
                } else {
#pragma unroll
                    for (int q = 0; q < 10; ++q)
                        w[q] = 0.f;
                    w[10] = __int_as_float(-2);
                }
#pragma unroll
                for (int q = 0; q < 11; ++q)
                    s_ibuf[q * ITILE + il] = w[q];
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            int il = k * TI + ti;
            const long long gi = TJ > 1 ? 0 : i_index(t, il);
            if constexpr (TJ > 1) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float hi = s_ibuf[d * ITILE + il], lo = s_ibuf[(3 + d) * ITILE + il];
                    const float w = -s_ibuf[(6 + d) * ITILE + il];
                    nxh[k][d] = make_float2(-hi, -hi);
                    nxl[k][d] = make_float2(-lo, -lo);
                    nv[k][d] = make_float2(w, w);
                }
                h2[k] = s_ibuf[9 * ITILE + il];
                iid[k] = __float_as_int(s_ibuf[10 * ITILE + il]);
            } else if (gi >= 0) {
                const g6x_irec &r = a.irec[gi];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    double x = r.x[d];
                    float hi = __double2float_rn(x);
                    float lo = __double2float_rn(x - (double)hi);
                    nxh[k][d] = make_float2(-hi, -hi);
                    nxl[k][d] = make_float2(-lo, -lo);
                    float w = -(float)r.v[d];
                    nv[k][d] = make_float2(w, w);
                }
                h2[k] = (float)(r.h2 + (double)eps2.x);
                iid[k] = r.index;
            } else {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    nxh[k][d] = make_float2(0.f, 0.f);
                    nxl[k][d] = make_float2(0.f, 0.f);
                    nv[k][d] = make_float2(0.f, 0.f);
                }
                h2[k] = 0.f;
                iid[k] = -2;
            }
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                ta[k][q] = make_float2(0.f, 0.f);
                cslot(k, q) = make_float2(0.f, 0.f);
            }
            tmin[k] = INF;
            nnr[k] = INF;
            nnt[k] = -1;
            nbn[k] = 0;
            tchk[k] = 0;
            nnc[k] = 0;
        }
        since_flush = 0;
        if constexpr (TJ > 1)
            __syncthreads();          // s_ibuf is reused by the next segment
    };

    // First j of the thread's share of tile nnt[k] whose key equals nnr[k],
    // recomputed with the loop's arithmetic (packed lanes round like the
    // scalar operations used here).  The loads of 8 j-particles are issued
    // together so the rescan costs a few memory latencies, not one per j.
    auto nn_rescan = [&](int k) -> int {
        if (!(nnr[k] < INF) || nnt[k] < 0)
            return -1;
        const float *T = a.pt + (size_t)nnt[k] * JW * JT;
        constexpr int CH = NNC ? CHP : 4;           // j-pairs loaded together
        const int kb = NNC ? nnc[k] * CH : 0, ke = NNC ? kb + CH : PPT;
        for (int kk0 = kb; kk0 < ke; kk0 += CH) {
            float key[2 * CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int kk = kk0 + u;
                    const int jj = 2 * (tj + kk * TJ) + h;
                    float r2u = INF;
                    int id = -1;
                    // FP: the tile was never stored; predict this j again
                    // with the same arithmetic (empty slots cannot win)
                    const int slot = nnt[k] * JT + jj;
                    if (kk < PPT && (!FP || slot < a.nj)) {
                        float ph[3], pl[3];
                        if constexpr (FP) {
                            const float hh = (float)(a.t_pred - js_t0(a.js, slot));
                            predict_ds_pos(hh, js_xds(a.js, slot), js_xds2(a.js, slot),
                                           js_v0m(a.js, slot), js_a2f(a.js, slot),
                                           js_j6f(a.js, slot), ph, pl);
                            id = js_idx(a.js, slot);
                        } else {
                            ph[0] = __ldg(T + W_XH * JT + jj);
                            ph[1] = __ldg(T + W_YH * JT + jj);
                            ph[2] = __ldg(T + W_ZH * JT + jj);
                            pl[0] = __ldg(T + W_XL * JT + jj);
                            pl[1] = __ldg(T + W_YL * JT + jj);
                            pl[2] = __ldg(T + W_ZL * JT + jj);
                            id = __float_as_int(__ldg(T + W_ID * JT + jj));
                        }
                        // the loop's own separation arithmetic, lane by lane
                        float dd[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if constexpr (DSS)
                                dd[d] = ds_sep1(ph[d], pl[d], nxh[k][d].x, nxl[k][d].x);
                            else
                                dd[d] = __fadd_rn(__fadd_rn(ph[d], nxh[k][d].x),
                                                  __fadd_rn(pl[d], nxl[k][d].x));
                        }
                        r2u = soft_r2(dd[0], dd[1], dd[2], eps2.x);
                    }
                    key[2 * u + h] = (id == iid[k]) ? INF : r2u;
                }
            }
#pragma unroll
            for (int u = 0; u < 2 * CH; ++u)
                if (key[u] == nnr[k])
                    return nnt[k] * JT + 2 * (tj + (kk0 + u / 2) * TJ) + (u & 1);
        }
        return -1;
    };

    // Reduction of i-tile t by the last CTA that finished it (Sect. 2.3:
    // partial forces are reduced on the GPU): every CTA that touched the tile
    // has written its partial records; P lanes per i-particle (P a power of
    // two, up to the warp, chosen from the number of segments) sum them in
    // FP64, combine by shuffles and pick the nearest neighbour (ties to the
    // lower j-slot); the launch uses this path only when a tile has few
    // partials, so the tail it adds is short.
    __shared__ int s_last;
    auto reduce_tile = [&](int t, long long clo, long long chi) {
        const int nseg = (int)(chi - clo + 1);
        int P = 1;
        while (P < 32 && 2 * P <= nseg)
            P *= 2;
        const int groups = NT / P;
        const int rounds = (ITILE + groups - 1) / groups;
        const int part = tid % P;
        for (int r = 0; r < rounds; ++r) {
            const int il = r * groups + tid / P;
            const long long gi = il < ITILE ? i_index(t, il) : -1;
            const bool valid = gi >= 0;
            float sh[7] = {0, 0, 0, 0, 0, 0, 0}, sl[7] = {0, 0, 0, 0, 0, 0, 0};
            float br = INF;
            int bj = -1;
            if (valid) {
                const PartialDS *PP = reinterpret_cast<const PartialDS *>(a.part);
#pragma unroll 4
                for (int q = part; q < nseg; q += P) {
                    const PartialDS *Pp = PP + (size_t)(clo + q + t) * ITILE + il;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float2 va = __ldcg(&Pp->acc[d]), vj = __ldcg(&Pp->jerk[d]);
                        ds_acc(sh[d], sl[d], va.x, va.y);
                        ds_acc(sh[3 + d], sl[3 + d], vj.x, vj.y);
                    }
                    const float2 vp = __ldcg(&Pp->pot);
                    ds_acc(sh[6], sl[6], vp.x, vp.y);
                    const float rr = __ldcg(&Pp->nnr2);
                    const int jj = __ldcg(&Pp->nnj);
                    if (jj >= 0 && (bj < 0 || rr < br || (rr == br && jj < bj))) {
                        br = rr;
                        bj = jj;
                    }
                }
            }
            for (int off = P / 2; off > 0; off >>= 1) {
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const float oh = __shfl_xor_sync(0xffffffffu, sh[q], off);
                    const float ol = __shfl_xor_sync(0xffffffffu, sl[q], off);
                    ds_acc(sh[q], sl[q], oh, ol);
                }
                const float rr = __shfl_xor_sync(0xffffffffu, br, off);
                const int jj = __shfl_xor_sync(0xffffffffu, bj, off);
                if (jj >= 0 && (bj < 0 || rr < br || (rr == br && jj < bj))) {
                    br = rr;
                    bj = jj;
                }
            }
            if (valid && part == 0) {
                g6x_out o;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    o.acc[d] = (double)sh[d] + (double)sl[d];
                    o.jerk[d] = (double)sh[3 + d] + (double)sl[3 + d];
                }
                o.pot = -((double)sh[6] + (double)sl[6]);
                o.nnb = bj >= 0 ? a.jidx[bj] : -1;
                o.nnr2 = bj >= 0 ? br : INF;
                a.out[gi] = o;
                if constexpr (LIST) {
                    // the list partials in segment order (ascending j),
                    // truncated at the list length; the count is the total
                    long long pos = 0, total = 0;
                    for (int q = 0; q < nseg; ++q) {
                        const size_t slot = (size_t)(clo + q + t) * ITILE + il;
                        const int cnt = __ldcg(&a.nbc[slot]);
                        const int kept = min(cnt, a.nbseg);
                        const int *src = a.nbl + slot * a.nbseg;
                        for (int e = 0; e < kept && pos + e < a.maxnb; ++e)
                            a.nbl_out[(size_t)gi * a.maxnb + pos + e] = a.jidx[__ldcg(&src[e])];
                        pos += kept;
                        total += cnt;
                    }
                    a.nblen_out[gi] = (int)min(total, (long long)INT_MAX);
                }
            }
        }
    };

    // After this CTA's partials of i-tile t are written: count it in; the
    // CTA that completes the count reduces the tile and resets the counter
    // for the next launch.  (A launch that gives up early leaves counts
    // behind; the host clears all counters after any reported error.)
    auto tile_done = [&](int t) {
        const long long clo = work_owner(g_start(t), W, G);
        const long long chi = work_owner(g_start(t + 1) - 1, W, G);
        // a batch line mixes entries of every span: only those with a few
        // partials are reduced here, the others by K3 (the same test there)
        if constexpr (BATCH)
            if (!fused_span(clo, chi, W, G))
                return;
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned need = (unsigned)(chi - clo + 1);
            const unsigned prev = atomicAdd(&a.tcnt[t], 1u);
            s_last = (prev + 1 == need) ? 1 : 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            reduce_tile(t, clo, chi);
            if (tid == 0)
                a.tcnt[t] = 0u;
        }
        __syncthreads();
    };

    // Where a thread's list entries for slot il of segment seg go: with whole
    // j-tiles per thread, the list partial itself; with TJ j-groups, the
    // group's own run (ascending j, as the group walks its j-pairs in
    // order), merged into the list partial when the segment ends.
    auto list_run = [&](long long seg, int il, int g) -> int * {
        if constexpr (LRUN)
            return a.nbr + (((size_t)seg * ITILE + il) * TJ + g) * a.nbseg;
        else
            return a.nbl + ((size_t)seg * ITILE + il) * a.nbseg;
    };

    auto finalize = [&](int t) {
        flush();
        const long long seg = c + t;
        PartialDS *PP = reinterpret_cast<PartialDS *>(a.part);
        if constexpr (TJ == 1) {
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                int il = k * TI + ti;
                PartialDS *P = PP + (size_t)seg * ITILE + il;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    P->acc[d] = cslot(k, d);
                    P->jerk[d] = cslot(k, 3 + d);
                }
                P->pot = cslot(k, 6);
                P->nnr2 = unsoftened(nnr[k], eps2.x);
                P->nnj = nn_rescan(k);
                if constexpr (LIST) {
                    a.nbc[(size_t)seg * ITILE + il] = nbn[k];
                    if (nbn[k] > 0)
                        atomicMax(a.nbmax, min(nbn[k], a.maxnb));
                }
            }
        } else {
            // The TJ j-groups of an i-particle combine in place: every
            // thread's compensated sums are in comp[], its nearest neighbour
            // goes to s_nnr / s_nnj, and one thread per i-particle adds the
            // groups in compensated FP32 (neighbour ties to the lower j-slot).
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                s_nnr[k * NT + tid] = nnr[k];
                s_nnj[k * NT + tid] = nn_rescan(k);
                if constexpr (LRUN)
                    s_nbn[k * NT + tid] = nbn[k];
            }
            __syncthreads();
            for (int il = tid; il < ITILE; il += NT) {
                const int k = il / TI, ii = il % TI;
                float sh[7], sl[7];
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    sh[q] = 0.f;
                    sl[q] = 0.f;
                }
                float br = INF;
                int bj = -1;
                for (int g = 0; g < TJ; ++g) {
                    const int o = g * TI + ii;
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        const float2 hl = comp[(k * 7 + q) * NT + o];
                        ds_acc(sh[q], sl[q], hl.x, hl.y);
                    }
                    const float r = s_nnr[k * NT + o];
                    const int jj = s_nnj[k * NT + o];
                    if (jj >= 0 && (r < br || (r == br && (bj < 0 || jj < bj)))) {
                        br = r;
                        bj = jj;
                    }
                }
                PartialDS *P = PP + (size_t)seg * ITILE + il;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    P->acc[d] = make_float2(sh[d], sl[d]);
                    P->jerk[d] = make_float2(sh[3 + d], sl[3 + d]);
                }
                P->pot = make_float2(sh[6], sl[6]);
                P->nnr2 = unsoftened(br, eps2.x);
                P->nnj = bj;
                if constexpr (LRUN) {
                    // merge the TJ ascending runs into the list partial;
                    // a run keeps its first nbseg entries, and a total above
                    // nbseg makes the host compute the lists again with more
                    // room, unless nbseg is already the list length (then
                    // the lowest maxnb j of the runs are the lowest overall)
                    int tot = 0;
                    for (int g = 0; g < TJ; ++g)
                        tot += s_nbn[k * NT + g * TI + ii];
                    const int keep = min(tot, a.nbseg);
                    if (keep > 0) {
                        int *dst = a.nbl + ((size_t)seg * ITILE + il) * a.nbseg;
                        for (int g = 0; g < TJ; ++g) {
                            const int o = k * NT + g * TI + ii;
                            s_nnj[o] = 0;               // read position in the run
                            s_nbh[o] = s_nbn[o] > 0 ? list_run(seg, il, g)[0] : INT_MAX;
                        }
                        for (int e = 0; e < keep; ++e) {
                            int best = INT_MAX, bg = 0;
                            for (int g = 0; g < TJ; ++g) {
                                const int h = s_nbh[k * NT + g * TI + ii];
                                if (h < best) {
                                    best = h;
                                    bg = g;
                                }
                            }
                            dst[e] = best;
                            const int o = k * NT + bg * TI + ii;
                            const int pos = ++s_nnj[o];
                            s_nbh[o] = pos < min(s_nbn[o], a.nbseg) ? list_run(seg, il, bg)[pos]
                                                                    : INT_MAX;
                        }
                    }
                    a.nbc[(size_t)seg * ITILE + il] = tot;
                    if (tot > 0)
                        atomicMax(a.nbmax, min(tot, a.maxnb));
                }
            }
            __syncthreads();
        }
        if (a.fused)
            tile_done(t);
    };

    // All pairs of the thread's share of one staged tile.  SELF: apply the
    // per-pair self test (tiles that may hold one of the i-particles).
    auto tile_pass = [&](const float *S, int t, int jt, auto self_tag) {
        constexpr bool SELF = decltype(self_tag)::value;
        const float2 *XH = reinterpret_cast<const float2 *>(S + W_XH * JT);
        const float2 *YH = reinterpret_cast<const float2 *>(S + W_YH * JT);
        const float2 *ZH = reinterpret_cast<const float2 *>(S + W_ZH * JT);
        const float2 *MM = reinterpret_cast<const float2 *>(S + W_M * JT);
        const float2 *XL = reinterpret_cast<const float2 *>(S + W_XL * JT);
        const float2 *YL = reinterpret_cast<const float2 *>(S + W_YL * JT);
        const float2 *ZL = reinterpret_cast<const float2 *>(S + W_ZL * JT);
        const float2 *VX = reinterpret_cast<const float2 *>(S + W_VX * JT);
        const float2 *VY = reinterpret_cast<const float2 *>(S + W_VY * JT);
        const float2 *VZ = reinterpret_cast<const float2 *>(S + W_VZ * JT);
        const int2 *ID = reinterpret_cast<const int2 *>(S + W_ID * JT);
        // j-pair kk of the thread's share against its NI i-particles; mins[k]
        // receives the smaller key
        auto jpair = [&](int kk, float (&mins)[NI]) {
            const int jp = tj + kk * TJ;
            const float2 xh = XH[jp], yh = YH[jp], zh = ZH[jp], mj = MM[jp];
            const float2 xl = XL[jp], yl = YL[jp], zl = ZL[jp];
            const float2 vx = VX[jp], vy = VY[jp], vz = VZ[jp];
            int2 id = make_int2(0, 0);
            if constexpr (SELF)
                id = ID[jp];
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                float2 dx, dy, dz;
                if constexpr (DSS) {
                    dx = ds_sep2(xh, xl, nxh[k][0], nxl[k][0]);
                    dy = ds_sep2(yh, yl, nxh[k][1], nxl[k][1]);
                    dz = ds_sep2(zh, zl, nxh[k][2], nxl[k][2]);
                } else {
                    dx = __fadd2_rn(__fadd2_rn(xh, nxh[k][0]), __fadd2_rn(xl, nxl[k][0]));
                    dy = __fadd2_rn(__fadd2_rn(yh, nxh[k][1]), __fadd2_rn(yl, nxl[k][1]));
                    dz = __fadd2_rn(__fadd2_rn(zh, nxh[k][2]), __fadd2_rn(zl, nxl[k][2]));
                }
                const float2 ux = __fadd2_rn(vx, nv[k][0]);
                const float2 uy = __fadd2_rn(vy, nv[k][1]);
                const float2 uz = __fadd2_rn(vz, nv[k][2]);
                float2 key = soft_r2(dx, dy, dz, eps2);
                if constexpr (SELF) {
                    key.x = (id.x == iid[k]) ? INF : key.x;
                    key.y = (id.y == iid[k]) ? INF : key.y;
                }
                float2 ri, ri2;
                ri.x = rsqrt_approx(key.x);
                ri.y = rsqrt_approx(key.y);
                ri2.x = rcp_approx(key.x);
                ri2.y = rcp_approx(key.y);
                const float2 rv = __ffma2_rn(dz, uz, __ffma2_rn(dy, uy, __fmul2_rn(dx, ux)));
                const float2 mr = __fmul2_rn(mj, ri);
                const float2 mr3 = __fmul2_rn(mr, ri2);
                const float2 sc = __fmul2_rn(__fmul2_rn(rv, ri2), m3);
                ta[k][6] = __fadd2_rn(ta[k][6], mr);
                ta[k][0] = __ffma2_rn(mr3, dx, ta[k][0]);
                ta[k][1] = __ffma2_rn(mr3, dy, ta[k][1]);
                ta[k][2] = __ffma2_rn(mr3, dz, ta[k][2]);
                ta[k][3] = __ffma2_rn(mr3, __ffma2_rn(sc, dx, ux), ta[k][3]);
                ta[k][4] = __ffma2_rn(mr3, __ffma2_rn(sc, dy, uy), ta[k][4]);
                ta[k][5] = __ffma2_rn(mr3, __ffma2_rn(sc, dz, uz), ta[k][5]);
                mins[k] = fminf(mins[k], fminf(key.x, key.y));
            }
        };
        // Lists: the entries of chunk ch against i-particle k, the keys
        // computed again with the loop's arithmetic (packed lanes round like
        // the scalar operations used here), in ascending j.  Called only for
        // chunks whose smallest key is below the radius, so the pair loop
        // itself carries no list test.
        auto list_chunk = [&](int ch, int k) {
            int *dst = list_run(c + t, k * TI + ti, tj);
            for (int u = 0; u < CHP; ++u) {
                const int jp = tj + (ch * CHP + u) * TJ;
                const float2 xh = XH[jp], yh = YH[jp], zh = ZH[jp];
                const float2 xl = XL[jp], yl = YL[jp], zl = ZL[jp];
                const int2 id = ID[jp];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float dd[3];
                    const float xs[3] = {h ? xh.y : xh.x, h ? yh.y : yh.x, h ? zh.y : zh.x};
                    const float xt[3] = {h ? xl.y : xl.x, h ? yl.y : yl.x, h ? zl.y : zl.x};
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        if constexpr (DSS)
                            dd[d] = ds_sep1(xs[d], xt[d], nxh[k][d].x, nxl[k][d].x);
                        else
                            dd[d] = __fadd_rn(__fadd_rn(xs[d], nxh[k][d].x),
                                              __fadd_rn(xt[d], nxl[k][d].x));
                    }
                    float key = soft_r2(dd[0], dd[1], dd[2], eps2.x);
                    if ((h ? id.y : id.x) == iid[k])
                        key = INF;
                    if (key < h2[k]) {
                        if (nbn[k] < a.nbseg)
                            dst[nbn[k]] = jt * JT + 2 * jp + h;
                        ++nbn[k];
                    }
                }
            }
        };
        if constexpr (NNC || LIST) {
            for (int ch = 0; ch < PPT / CHP; ++ch) {
                float cm[NI];
#pragma unroll
                for (int k = 0; k < NI; ++k)
                    cm[k] = INF;
#pragma unroll UNR
                for (int u = 0; u < CHP; ++u)
                    jpair(ch * CHP + u, cm);
#pragma unroll
                for (int k = 0; k < NI; ++k) {
                    if constexpr (LIST)
                        if (cm[k] < h2[k])
                            list_chunk(ch, k);
                    if (cm[k] < tmin[k]) {      // the first chunk that reaches the minimum
                        tmin[k] = cm[k];
                        tchk[k] = ch;
                    }
                }
            }
        } else {
#pragma unroll UNR
            for (int kk = 0; kk < PPT; ++kk)
                jpair(kk, tmin);
        }
    };

    int cur_g = g_of(wb);
    for (int q = 0; q < ntile; ++q) {
        const long long p = wb + q;
        while (g_start(cur_g + 1) <= p)
            ++cur_g;
        const int t = cur_g;
        const int jt = jt_of(p, t);
        if (t != cur_t) {
            if (cur_t >= 0)
                finalize(cur_t);
            load_i(t);
            cur_t = t;
        }
        const int s = q % NS;
        const uint32_t par = (uint32_t)((q / NS) & 1);
        // Does this tile hold the j-particle of one of the warp's i-particles?
        auto self_test = [&](int2 rg) -> bool {
            bool mine = false;
#pragma unroll
            for (int k = 0; k < NI; ++k)
                mine |= (iid[k] >= rg.x && iid[k] <= rg.y);
            return __any_sync(0xffffffffu, mine);
        };
        auto pairs_of_tile = [&](const float *S, bool self_tile) {
            if (self_tile)
                tile_pass(S, t, jt, std::true_type{});
            else
                tile_pass(S, t, jt, std::false_type{});
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                if (tmin[k] < nnr[k]) {
                    nnr[k] = tmin[k];
                    nnt[k] = jt;
                    nnc[k] = tchk[k];
                }
                tmin[k] = INF;
            }
            if (++since_flush >= FLUSH) {
                flush();
                since_flush = 0;
            }
        };
        // Give up: wait (bounded, always the full limit) for this CTA's
        // copies still in flight so none lands in shared memory after exit,
        // then report.
        auto give_up = [&]() {
            if (tid == 0) {
                for (int r = q; r < q + NS && r < ntile; ++r)
                    mbar_wait_bounded(&bar[r % NS], (uint32_t)((r / NS) & 1),
                                      WAIT_LIMIT_NS);
                *(volatile int *)a.err = G6_ETIMEDOUT;
            }
        };
        if constexpr (FP) {
            const bool ready = mbar_wait_bounded(&bar[s], par, a.wait_ns);
            if (!ready)
                s_abort = 1;
            else
                predict_tile(s, jt);
            __syncthreads();
            if (s_abort) {
                give_up();
                return;
            }
            if (tid == 0 && q + NS < ntile)
                issue(q + NS);               // the raw stage is free again
            int2 rg = make_int2(INT_MAX, -1);
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
                rg.x = min(rg.x, s_wlo[w]);
                rg.y = max(rg.y, s_whi[w]);
            }
            pairs_of_tile(pbuf, self_test(rg));
            __syncthreads();                     // pbuf is rewritten by the next tile
        } else {
            const bool self_tile = self_test(a.trange[jt]);
            const bool ready = mbar_wait_bounded(&bar[s], par, a.wait_ns);
            if (!ready)
                s_abort = 1;
            else
                pairs_of_tile(stage_buf + (size_t)s * JW * JT, self_tile);
            __syncthreads();
            if (s_abort) {
                give_up();
                return;
            }
            if (tid == 0 && q + NS < ntile)
                issue(q + NS);
        }
    }
    finalize(cur_t);
}

// The same pair sum entirely in FP64, one i-particle per thread, j-tiles
// staged in shared memory by plain cooperative loads.
template <bool LIST>
__global__ void __launch_bounds__(128) k_force_64(const ForceArgs a)
{
    grid_dep_wait();                // the FP64 prediction (see k_force_ds)
    grid_dep_launch();
    constexpr int TI = 128;
    __shared__ double4_32a sp[JT], sv[JT];
    const int tid = threadIdx.x;
    const long long G = gridDim.x, c = blockIdx.x;
    const long long wb = work_begin(c, a.W, G), we = work_begin(c + 1, a.W, G);
    if (we <= wb)
        return;
    double xi[3] = {0, 0, 0}, vi[3] = {0, 0, 0}, h2 = 0.0;
    int iid = -2;
    double s[7];
    double nnr = 0.0;
    int nnj = -1, nbn = 0;
    int cur_t = -1;
    const double INF = __longlong_as_double(0x7ff0000000000000ll);

    auto finalize = [&](int t) {
        const long long seg = c + t;
        Partial64 *P = reinterpret_cast<Partial64 *>(a.part) + (size_t)seg * TI + tid;
        for (int d = 0; d < 3; ++d) {
            P->acc[d] = s[d];
            P->jerk[d] = s[3 + d];
        }
        P->pot = s[6];
        P->nnr2 = nnr;
        P->nnj = nnj;
        if constexpr (LIST) {
            a.nbc[(size_t)seg * TI + tid] = nbn;
            if (nbn > 0)
                atomicMax(a.nbmax, min(nbn, a.maxnb));
        }
    };

    for (long long p = wb; p < we; ++p) {
        const int t = (int)(p / a.J);
        const int jt = (int)(p - (long long)t * a.J);
        if (t != cur_t) {
            if (cur_t >= 0)
                finalize(cur_t);
            long long gi = (long long)t * TI + tid;
            if (gi < a.ni) {
                const g6x_irec &r = a.irec[gi];
                for (int d = 0; d < 3; ++d) {
                    xi[d] = r.x[d];
                    vi[d] = r.v[d];
                }
                h2 = r.h2;
                iid = r.index;
            } else {
                iid = -2;
            }
            for (int q = 0; q < 7; ++q)
                s[q] = 0.0;
            nnr = INF;
            nnj = -1;
            nbn = 0;
            cur_t = t;
        }
        __syncthreads();
        for (int k = tid; k < JT; k += TI) {
            sp[k] = a.p64[(size_t)jt * JT + k];
            sv[k] = a.v64[(size_t)jt * JT + k];
        }
        __syncthreads();
        const int jbase = jt * JT;
        for (int jj = 0; jj < JT; ++jj) {
            const double4_32a pj = sp[jj], vj = sv[jj];
            const double dx = pj.x - xi[0], dy = pj.y - xi[1], dz = pj.z - xi[2];
            const double ux = vj.x - vi[0], uy = vj.y - vi[1], uz = vj.z - vi[2];
            const double r2u = dx * dx + dy * dy + dz * dz;
            const double key = ((int)vj.w == iid) ? INF : r2u;
            const double ri = rsqrt(key + a.eps2);
            const double rv = dx * ux + dy * uy + dz * uz;
            const double ri2 = ri * ri;
            const double mr = pj.w * ri;
            const double mr3 = mr * ri2;
            const double sc = -3.0 * rv * ri2;
            s[6] += mr;
            s[0] += mr3 * dx;
            s[1] += mr3 * dy;
            s[2] += mr3 * dz;
            s[3] += mr3 * (ux + sc * dx);
            s[4] += mr3 * (uy + sc * dy);
            s[5] += mr3 * (uz + sc * dz);
            if (key < nnr) {
                nnr = key;
                nnj = jbase + jj;
            }
            if constexpr (LIST) {
                if (key < h2) {
                    if (nbn < a.nbseg)
                        a.nbl[((size_t)(c + t) * TI + tid) * a.nbseg + nbn] = jbase + jj;
                    ++nbn;
                }
            }
        }
    }
    finalize(cur_t);
}

// ----------------------------------------------------------------- K3 ---

struct ReduceArgs {
    const void *part;                 // PartialDS or Partial64
    const int *nbl, *nbc;
    const int *jidx;
    g6x_out *out;
    int *nbl_out, *nblen_out;
    long long W;
    int J, G, ni, itile, list;
    int maxnb, nbseg;                 // list length kept; entries per list partial
    int fused;                        // batch: entries with few partials were reduced by K2
};


// K3, one warp per i-particle: lanes take the partials of the CTAs that
// touched its i-tile and combine with warp shuffles (Sect. 2.3, 2.5).
// Neighbour lists are concatenated in segment order, which is ascending j,
// and truncated at the context's list length (Sect. 4).
template <class PT>
__global__ void __launch_bounds__(256) k_reduce(const ReduceArgs a)
{
    grid_dep_wait();                // the partials of the force kernel
    const int lane = threadIdx.x & 31;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= a.ni)
        return;
    const PT *part = reinterpret_cast<const PT *>(a.part);
    const int t = (int)(i / a.itile), il = (int)(i % a.itile);
    const long long p0 = (long long)t * a.J, p1 = p0 + a.J;
    const long long clo = work_owner(p0, a.W, a.G), chi = work_owner(p1 - 1, a.W, a.G);
    PartialSum<PT> acc;
    acc.init();
#pragma unroll 4
    for (long long cc = clo + lane; cc <= chi; cc += 32)
        acc.add(part[(size_t)(cc + t) * a.itile + il]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        acc.shfl_combine(off);
    if (lane == 0)
        a.out[i] = result_of(acc, a.jidx);
    if (!a.list)
        return;
    long long base = 0, total = 0;
    for (long long c0 = clo; c0 <= chi; c0 += 32) {
        long long cc = c0 + lane;
        int cnt = cc <= chi ? a.nbc[(size_t)(cc + t) * a.itile + il] : 0;
        int kept = min(cnt, a.nbseg);
        int incl = kept;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off)
                incl += v;
        }
        long long pos0 = base + incl - kept;
        const int *src = a.nbl + ((size_t)(cc + t) * a.itile + il) * a.nbseg;
        for (int e = 0; e < kept && pos0 + e < a.maxnb; ++e)
            a.nbl_out[(size_t)i * a.maxnb + pos0 + e] = a.jidx[src[e]];
        long long ctot = cnt;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            ctot += __shfl_xor_sync(0xffffffffu, ctot, off);
        total += ctot;
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0)
        a.nblen_out[i] = (int)min(total, (long long)INT_MAX);
}

// K3 for blocks whose i-tiles were split over many CTAs (small m): one CTA
// of 256 threads per i-particle, the partials strided over all its threads,
// combined by warp shuffles and then across the 8 warps.  No lists.
template <class PT>
__global__ void __launch_bounds__(256) k_reduce_wide(const ReduceArgs a)
{
    grid_dep_wait();                // the partials of the force kernel
    const long long i = blockIdx.x;
    if (i >= a.ni)
        return;
    const PT *part = reinterpret_cast<const PT *>(a.part);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = (int)(i / a.itile), il = (int)(i % a.itile);
    const long long p0 = (long long)t * a.J, p1 = p0 + a.J;
    const long long clo = work_owner(p0, a.W, a.G), chi = work_owner(p1 - 1, a.W, a.G);
    PartialSum<PT> acc;
    acc.init();
#pragma unroll 4
    for (long long cc = clo + tid; cc <= chi; cc += 256)
        acc.add(part[(size_t)(cc + t) * a.itile + il]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        acc.shfl_combine(off);
    __shared__ PartialSum<PT> ws[8];
    if (lane == 0)
        ws[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        if (lane < 8)
            acc = ws[lane];
        else
            acc.init();
#pragma unroll
        for (int off = 4; off > 0; off >>= 1)
            acc.shfl_combine(off);
        if (lane == 0)
            a.out[i] = result_of(acc, a.jidx);
    }
    if (!a.list)
        return;
    // Lists: the partials' entries in segment order (ascending j), 256
    // partials per pass, each placed by a block-wide scan of the counts
    // kept; truncated at the list length, the total count kept apart.
    __shared__ int s_kept[8];
    __shared__ long long s_cnt[8];
    long long base = 0, total = 0;
    for (long long c0 = clo; c0 <= chi; c0 += 256) {
        const long long cc = c0 + tid;
        const int cnt = cc <= chi ? a.nbc[(size_t)(cc + t) * a.itile + il] : 0;
        const int kept = min(cnt, a.nbseg);
        int incl = kept;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off)
                incl += v;
        }
        long long ctot = cnt;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            ctot += __shfl_xor_sync(0xffffffffu, ctot, off);
        __syncthreads();                    // the previous pass has read s_kept
        if (lane == 31)
            s_kept[warp] = incl;
        if (lane == 0)
            s_cnt[warp] = ctot;
        __syncthreads();
        int woff = 0, pass_kept = 0;
        long long pass_cnt = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            woff += w < warp ? s_kept[w] : 0;
            pass_kept += s_kept[w];
            pass_cnt += s_cnt[w];
        }
        const long long pos0 = base + woff + incl - kept;
        const int *src = a.nbl + ((size_t)(cc + t) * a.itile + il) * a.nbseg;
        for (int e = 0; e < kept && pos0 + e < a.maxnb; ++e)
            a.nbl_out[(size_t)i * a.maxnb + pos0 + e] = a.jidx[src[e]];
        base += pass_kept;
        total += pass_cnt;
    }
    if (tid == 0)
        a.nblen_out[i] = (int)min(total, (long long)INT_MAX);
}

// K3 for a batch: one warp per (global i-tile, slot) with an active
// i-particle; the CTAs that touched the i-tile follow from its work range.
template <class PT>
__global__ void __launch_bounds__(256) k_reduce_batch(const ReduceArgs a, BatchTables bt)
{
    const int lane = threadIdx.x & 31;
    const long long W = bt.hdr[0];
    const long long ngt = bt.hdr[1];
    const BatchGT *gt = bt.gt + bt.hdr[2];
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const PT *part = reinterpret_cast<const PT *>(a.part);
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
         w < ngt * a.itile; w += nwarps) {
        const int g = (int)(w / a.itile), il = (int)(w % a.itile);
        const int k = gt[g].cluster;
        const int li = gt[g].itile * a.itile + il;
        if (li >= bt.cl_ni[k])
            continue;                                  // uniform within the warp
        const long long clo = work_owner(gt[g].start, W, a.G);
        const long long chi = work_owner(gt[g + 1].start - 1, W, a.G);
        if (a.fused && fused_span(clo, chi, W, a.G))
            continue;                                  // reduced by the force kernel
        PartialSum<PT> acc;
        acc.init();
#pragma unroll 4
        for (long long cc = clo + lane; cc <= chi; cc += 32)
            if (work_begin(cc, W, a.G) < work_begin(cc + 1, W, a.G))   // CTA had work
                acc.add(part[(size_t)(cc + g) * a.itile + il]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            acc.shfl_combine(off);
        if (lane == 0)
            a.out[(long long)bt.cl_ioff[k] + li] = result_of(acc, a.jidx);
    }
}

// Limit of each wait for a staged j-tile in the force kernels (the drain of
// copies still in flight after a timeout always allows WAIT_LIMIT_NS).
unsigned long long g_wait_ns = WAIT_LIMIT_NS;

// A wait that nothing completes: one thread waits, with the same bounded
// wait as the force kernels, on an mbarrier that expects one arrival that
// never comes, and reports G6_ETIMEDOUT in the error word as they do.
__global__ void k_wait_probe(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0)
        return;
    mbar_init(&bar, 1);
    fence_barrier_init();
    if (!mbar_wait_bounded(&bar, 0, limit_ns))
        *(volatile int *)err = G6_ETIMEDOUT;
}

// ------------------------------------------------------------ variants ---

namespace {

using ForceFn = void (*)(const ForceArgs);

struct Variant {
    VariantInfo info;
    ForceFn fn;
    int threads;
    int smem;
};

// dynamic shared memory of a DS variant: NSTAGE j-tiles + compensated sums
constexpr int ds_smem(int nt, int ni)
{
    return NSTAGE * JW * JT * (int)sizeof(float) + ni * 7 * nt * (int)sizeof(float2);
}

// ... with fused prediction: FP_NSTAGE raw tiles + one predicted tile + sums
constexpr int fp_smem(int nt, int ni)
{
    return FP_NSTAGE * (int)RAW_TILE_BYTES + JW * JT * (int)sizeof(float)
           + ni * 7 * nt * (int)sizeof(float2);
}

const Variant kVariants[] = {
    {{128, 1, 2, 0, G6X_PREC_DS}, k_force_ds<128, 1, 2, false, 3, 2>, 128, ds_smem(128, 2)},
    {{128, 1, 1, 0, G6X_PREC_DS}, k_force_ds<128, 1, 1, false>, 128, ds_smem(128, 1)},
    {{64, 4, 1, 0, G6X_PREC_DS}, k_force_ds<64, 4, 1, false>, 256, ds_smem(256, 1)},
    {{32, 8, 1, 0, G6X_PREC_DS}, k_force_ds<32, 8, 1, false>, 256, ds_smem(256, 1)},
    {{16, 16, 1, 0, G6X_PREC_DS}, k_force_ds<16, 16, 1, false>, 256, ds_smem(256, 1)},
    {{128, 1, 1, 1, G6X_PREC_DS}, k_force_ds<128, 1, 1, true>, 128, ds_smem(128, 1)},
    {{32, 1, 1, 1, G6X_PREC_DS}, k_force_ds<32, 1, 1, true>, 32, ds_smem(32, 1)},
    {{128, 1, 1, 0, G6X_PREC_FP64}, k_force_64<false>, 128, 0},
    {{128, 1, 1, 1, G6X_PREC_FP64}, k_force_64<true>, 128, 0},
    // alternative shapes, for tuning
    {{128, 1, 2, 0, G6X_PREC_DS}, k_force_ds<128, 1, 2, false, 4, 2>, 128, ds_smem(128, 2)},
    {{128, 1, 2, 0, G6X_PREC_DS}, k_force_ds<128, 1, 2, false, 3, 4>, 128, ds_smem(128, 2)},
    {{128, 1, 3, 0, G6X_PREC_DS}, k_force_ds<128, 1, 3, false, 2, 2>, 128, ds_smem(128, 3)},
    {{96, 1, 2, 0, G6X_PREC_DS}, k_force_ds<96, 1, 2, false, 4, 2>, 96, ds_smem(96, 2)},
    // split-j shapes with two i-particles per thread, for small blocks
    {{8, 32, 2, 0, G6X_PREC_DS}, k_force_ds<8, 32, 2, false, 2, 2>, 256, ds_smem(256, 2)},
    {{16, 16, 2, 0, G6X_PREC_DS}, k_force_ds<16, 16, 2, false, 2, 2>, 256, ds_smem(256, 2)},
    {{32, 8, 2, 0, G6X_PREC_DS}, k_force_ds<32, 8, 2, false, 2, 2>, 256, ds_smem(256, 2)},
    {{64, 4, 2, 0, G6X_PREC_DS}, k_force_ds<64, 4, 2, false, 2, 2>, 256, ds_smem(256, 2)},
    // fused prediction (Eq. 1, Eq. 2 inside the force kernel, no separate
    // predictor launch) for small blocks: twins of variants 4, 14, 15, 16
    {{16, 16, 1, 0, G6X_PREC_DS, 1, 4}, k_force_ds<16, 16, 1, false, 1, 2, false, true>, 256,
     fp_smem(256, 1)},
    {{16, 16, 2, 0, G6X_PREC_DS, 1, 14}, k_force_ds<16, 16, 2, false, 2, 2, false, true>, 256,
     fp_smem(256, 2)},
    {{32, 8, 2, 0, G6X_PREC_DS, 1, 15}, k_force_ds<32, 8, 2, false, 2, 2, false, true>, 256,
     fp_smem(256, 2)},
    {{64, 4, 2, 0, G6X_PREC_DS, 1, 16}, k_force_ds<64, 4, 2, false, 2, 2, false, true>, 256,
     fp_smem(256, 2)},
    // full DS subtraction for the separations (accuracy ablation)
    {{128, 1, 2, 0, G6X_PREC_DS_DSSUB}, k_force_ds<128, 1, 2, false, 3, 2, false, false, true>,
     128, ds_smem(128, 2)},
    {{16, 16, 1, 0, G6X_PREC_DS_DSSUB}, k_force_ds<16, 16, 1, false, 1, 2, false, false, true>,
     256, ds_smem(256, 1)},
    // neighbour lists: the twins of variants 9, 4, 14, 15 and 16
    {{128, 1, 2, 1, G6X_PREC_DS}, k_force_ds<128, 1, 2, true, 4, 2>, 128, ds_smem(128, 2)},
    {{16, 16, 1, 1, G6X_PREC_DS}, k_force_ds<16, 16, 1, true, 2, 2>, 256, ds_smem(256, 1)},
    {{16, 16, 2, 1, G6X_PREC_DS}, k_force_ds<16, 16, 2, true, 2, 2>, 256, ds_smem(256, 2)},
    {{32, 8, 2, 1, G6X_PREC_DS}, k_force_ds<32, 8, 2, true, 2, 2>, 256, ds_smem(256, 2)},
    {{64, 4, 2, 1, G6X_PREC_DS}, k_force_ds<64, 4, 2, true, 2, 2>, 256, ds_smem(256, 2)},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

// Batch force kernels: the same pair loop over the batch work geometry.
const Variant kBatchVariants[] = {
    {{16, 16, 1, 0, G6X_PREC_DS}, k_force_ds<16, 16, 1, false, 1, 2, true>, 256, ds_smem(256, 1)},
    {{16, 16, 2, 0, G6X_PREC_DS}, k_force_ds<16, 16, 2, false, 2, 2, true>, 256, ds_smem(256, 2)},
    {{32, 8, 2, 0, G6X_PREC_DS}, k_force_ds<32, 8, 2, false, 2, 2, true>, 256, ds_smem(256, 2)},
    {{64, 4, 2, 0, G6X_PREC_DS}, k_force_ds<64, 4, 2, false, 2, 2, true>, 256, ds_smem(256, 2)},
    {{128, 1, 2, 0, G6X_PREC_DS}, k_force_ds<128, 1, 2, false, 3, 2, true>, 128, ds_smem(128, 2)},
    {{8, 32, 1, 0, G6X_PREC_DS}, k_force_ds<8, 32, 1, false, 1, 2, true>, 256, ds_smem(256, 1)},
    {{8, 32, 2, 0, G6X_PREC_DS}, k_force_ds<8, 32, 2, false, 2, 2, true>, 256, ds_smem(256, 2)},
    {{4, 64, 2, 0, G6X_PREC_DS}, k_force_ds<4, 64, 2, false, 2, 2, true>, 256, ds_smem(256, 2)},
};
constexpr int kNumBatchVariants = (int)(sizeof(kBatchVariants) / sizeof(kBatchVariants[0]));
int g_bocc[kNumBatchVariants];

int g_occ[kNumVariants];
bool g_smem_set[kNumVariants];

// Every kernel of the library asks for the same L1 / shared-memory split
// (the most shared memory), so consecutive launches never wait for an SM to
// re-divide its on-chip memory.
template <class F>
void pin_carveout(F *fn)
{
    static bool done = false;      // one flag per kernel (per template instance)
    if (!done) {
        cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaGetLastError();
        done = true;
    }
}

cudaError_t prepare_variant(int v)
{
    if (!g_smem_set[v]) {
        // static + dynamic shared memory may exceed the 48 KB default
        if (kVariants[v].smem > 0) {
            cudaError_t e = cudaFuncSetAttribute(
                kVariants[v].fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                kVariants[v].smem);
            if (e != cudaSuccess)
                return e;
        }
        cudaFuncSetAttribute(reinterpret_cast<const void *>(kVariants[v].fn),
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaGetLastError();
        g_smem_set[v] = true;
    }
    return cudaSuccess;
}

}  // namespace

int variant_count() { return kNumVariants + ws_variant_count(); }

VariantInfo variant_info(int v)
{
    return v < kNumVariants ? kVariants[v].info : ws_variant_info(v - kNumVariants);
}

int variant_occupancy(int v)
{
    if (v >= kNumVariants)
        return ws_variant_occupancy(v - kNumVariants);
    if (v < 0)
        return 0;
    if (g_occ[v] == 0) {
        if (prepare_variant(v) != cudaSuccess)
            return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &n, kVariants[v].fn, kVariants[v].threads, kVariants[v].smem) != cudaSuccess)
            return 0;
        g_occ[v] = n;
    }
    return g_occ[v];
}

// ------------------------------------------------------------- tuning ---
//
// Best (variant, grid multiplier) per precision and power-of-two block size,
// filled by the autotuner (g6x_autotune) or loaded from its file.  Grid =
// multiplier x SMs x resident CTAs per SM.  Buckets above the largest tuned
// one reuse that one.

namespace {
struct TuneEntry {
    int variant = -1;
    int gmul = 1;
};
TuneEntry g_tune[2][TUNE_BUCKETS];
}  // namespace

int tune_bucket(int ni)
{
    int b = 0;
    while (b < TUNE_BUCKETS - 1 && (2 << b) <= ni)
        ++b;
    return b;
}

void tune_set(int prec, int bucket, int variant, int gmul)
{
    if (prec < 0 || prec > 1 || bucket < 0 || bucket >= TUNE_BUCKETS)
        return;
    g_tune[prec][bucket].variant = variant;
    g_tune[prec][bucket].gmul = gmul < 1 ? 1 : gmul;
}

bool tune_get(int prec, int bucket, int *variant, int *gmul)
{
    if (prec < 0 || prec > 1 || bucket < 0 || bucket >= TUNE_BUCKETS)
        return false;
    int b = -1;
    if (g_tune[prec][bucket].variant >= 0) {
        b = bucket;
    } else {
        int top = -1;
        for (int q = 0; q < TUNE_BUCKETS; ++q)
            if (g_tune[prec][q].variant >= 0)
                top = q;
        if (top >= 0 && bucket > top)
            b = top;
    }
    if (b < 0)
        return false;
    *variant = g_tune[prec][b].variant;
    *gmul = g_tune[prec][b].gmul;
    return true;
}

bool tune_exact(int prec, int bucket, int *variant, int *gmul)
{
    if (prec < 0 || prec > 1 || bucket < 0 || bucket >= TUNE_BUCKETS
        || g_tune[prec][bucket].variant < 0)
        return false;
    *variant = g_tune[prec][bucket].variant;
    *gmul = g_tune[prec][bucket].gmul;
    return true;
}

void tune_clear()
{
    for (auto &row : g_tune)
        for (auto &e : row)
            e = TuneEntry();
}

namespace {

// Blocks the built-in choice gives the small-block kernel.  Measured on
// GB300 as the host wall time of a block step through the GRAPE calls
// (the separate predictor and split-j shapes overlap their three launches):
// faster for m <= 16 at every N (N = 131072, m = 16: 36 against 42 us);
// for m <= 32 once the j-set has 512 tiles (N = 32768: a tie; N = 2^20:
// 92 against 122 us); for m <= 64 only from about 1500 tiles on (N =
// 262144: 72 against 67 us; N = 2^20: 142 against 173 us); never above.
constexpr int WS_ANY_N_MAX_NI = 16;
constexpr int WS_MID_MAX_NI = 32;
constexpr long long WS_MID_MIN_JTILES = 512;
constexpr int WS_DEFAULT_MAX_NI = 64;
constexpr long long WS_MIN_JTILES = 2048;

// The built-in launch choice for a block of ni against nj_pad j-particles
// (no tuning table); *gmul receives the grid multiplier.
int heuristic_variant(int prec, int ni, int nj_pad, int list, bool allow_ws, int *gmul)
{
    *gmul = 1;
    if (prec == G6X_PREC_FP64)
        return list ? 8 : 7;
    if (prec == G6X_PREC_DS_DSSUB && !list) {
        *gmul = ni > 2048 ? 2 : 1;
        return ni <= 32 ? 22 : 21;
    }
    if (allow_ws && !list
        && (ni <= WS_ANY_N_MAX_NI
            || (ni <= WS_MID_MAX_NI && nj_pad / JT >= WS_MID_MIN_JTILES)
            || (ni <= WS_DEFAULT_MAX_NI && nj_pad / JT >= WS_MIN_JTILES))) {
        // the warp-specialised small-block kernel: the narrowest i-tile
        // (one i-particle per thread) that holds the whole block
        int best = -1, best_tile = INT_MAX;
        for (int k = 0; k < ws_variant_count(); ++k) {
            const VariantInfo w = ws_variant_info(k);
            const int tile = w.ti * w.nper;
            if (w.nper == 1 && tile >= ni && tile < best_tile) {
                best = k;
                best_tile = tile;
            }
        }
        if (best >= 0)
            return kNumVariants + best;
    }
    // The widest i-tile the block size allows, narrowed while the work
    // line would hold too few (i-tile, j-tile) units for the SMs: wide
    // tiles need many j-tiles to keep every CTA busy, so small j-sets
    // take narrower tiles at the same m.  (The 256-wide tile from 65536
    // units on, measured with Plummer spheres: at N = 131072 the 128-wide
    // split-j tile is 9 % faster for m = 8192 and 2 % for m = 32768, the
    // wide one 4 % faster for m = 65536; at N = 32768, m = N the split-j
    // tile is 16 % faster; at N = 2^20, m = 4096 the wide one by 1 %.)
    struct Shape {
        int v, itile, max_ni;
        long long min_units;
    };
    static constexpr Shape plain_shapes[] = {
        {9, 256, INT_MAX, 65536},  // 128 threads, two i each, whole j-tiles, 4 CTAs per SM
        {16, 128, 2048, 4096},     // 64 x 4 threads, two i each
        {15, 64, 128, 2048},       // 32 x 8 threads, two i each
        {14, 32, 64, 2048},        // 16 x 16 threads, two i each
        {4, 16, 32, 0},            // 16 x 16 threads, one i each
    };
    // their twins with neighbour lists (the wide shape only on long work
    // lines: at N = 131072 the 64 x 4 twin is 6 % faster for m = 16384 and
    // 4 % for m = 65536, where the plain wide shape is the faster one)
    static constexpr Shape list_shapes[] = {
        {23, 256, INT_MAX, 1LL << 18},
        {27, 128, 2048, 4096},
        {26, 64, 128, 2048},
        {25, 32, 64, 2048},
        {24, 16, 32, 0},
    };
    const Shape *shapes = list ? list_shapes : plain_shapes;
    const long long jtl = nj_pad / JT;
    int k = 0;
    while (shapes[k].min_units > 0
           && (ni <= shapes[k + 1].max_ni
               || (long long)((ni + shapes[k].itile - 1) / shapes[k].itile) * jtl
                      < shapes[k].min_units))
        ++k;
    *gmul = 1;
    if (shapes[k].v == 9 || shapes[k].v == 23) {
        // Several waves of CTAs per SM: the warp schedulers favour the
        // oldest CTAs, so equal shares of the work line finish at different
        // times, and with one wave the SMs run their last stretch with few
        // warps.  Later waves fill those slots.  More CTAs also mean more
        // partial records and i-tile loads, so the count follows the length
        // of the work line (measured at N = 2^20: 1, 2, 2, 4, 8 waves best
        // for m = 4096, 16384, 65536, 262144, 2^20).
        const long long units = (long long)((ni + 255) / 256) * jtl;
        *gmul = units < (1LL << 18) ? 1 : units < (1LL << 21) ? 2 : units < (1LL << 23) ? 4 : 8;
    }
    return shapes[k].v;
}

}  // namespace

// Whether the built-in choice may take the warp-specialised small-block
// kernel (where the caller allows a fused prediction).
bool g_ws_default = true;

ForceConfig choose_config(int prec, int ni, int nj_pad, int list, int sm_count,
                          int force_variant, int force_grid, bool allow_fpred)
{
    const int nvar = variant_count();
    int v;
    int gmul = 1, tv = -1;
    if (force_variant < 0 && !list && tune_get(prec, tune_bucket(ni), &tv, &gmul)
        && tv >= 0 && tv < nvar && variant_info(tv).prec == prec && !variant_info(tv).list)
        force_variant = tv;
    else
        gmul = 1;
    if (force_variant >= 0 && force_variant < nvar)
        v = force_variant;
    else
        v = heuristic_variant(prec, ni, nj_pad, list, allow_fpred && g_ws_default, &gmul);
    // a fused-prediction shape only where the caller can use it (DS
    // predictor, the j-store current); otherwise its separate twin, or for
    // the small-block kernel (no twin; one i-tile) the built-in choice
    {
        const VariantInfo w = variant_info(v);
        if (w.fpred && (!allow_fpred || list || (w.ws && ni > w.ti * w.nper))) {
            if (w.twin >= 0)
                v = w.twin;
            else
                v = heuristic_variant(prec, ni, nj_pad, list, false, &gmul);
        }
    }
    const VariantInfo vi = variant_info(v);
    ForceConfig c{};
    c.variant = v;
    c.ti = vi.ti;
    c.tj = vi.tj;
    c.nper = vi.nper;
    c.itile = vi.ti * vi.nper;
    c.jtiles = nj_pad / JT;
    c.n_itile = (ni + c.itile - 1) / c.itile;
    c.work = (long long)c.n_itile * c.jtiles;
    c.smem = vi.ws ? ws_variant_smem(v - kNumVariants) : kVariants[v].smem;
    c.list = vi.list;
    c.prec = vi.prec;
    c.ws = vi.ws;
    int occ = variant_occupancy(v);
    if (occ < 1)
        occ = 1;
    long long g = force_grid > 0 ? force_grid : (long long)sm_count * occ * gmul;
    if (g > c.work)
        g = c.work;
    if (g < 1)
        g = 1;
    c.grid = (int)g;
    return c;
}

size_t partial_slots(const ForceConfig &cfg)
{
    if (cfg.ws)
        return ws_partial_slots(cfg.grid, cfg.itile);
    return (size_t)(cfg.grid + cfg.n_itile) * cfg.itile;
}

size_t list_part_ints(const ForceConfig &cfg, int nbseg)
{
    return partial_slots(cfg) * (size_t)nbseg * (cfg.tj > 1 ? 1 + cfg.tj : 1);
}

size_t counter_slots(const ForceConfig &cfg)
{
    if (cfg.ws) {
        const int gs = ws_group_size(cfg.grid);
        return (size_t)(cfg.grid + gs - 1) / gs + 1;
    }
    return (size_t)cfg.n_itile;
}

cudaError_t launch_init_store(JStore js, cudaStream_t s)
{
    int blocks = (js.cap + 255) / 256;
    if (blocks > 65535)
        blocks = 65535;
    pin_carveout(k_init_store);
    k_init_store<<<blocks, 256, 0, s>>>(js);
    return cudaGetLastError();
}

cudaError_t launch_irec_from_store(JStore js, g6x_irec *out, int m, cudaStream_t s)
{
    if (m <= 0)
        return cudaSuccess;
    pin_carveout(k_irec_from_store);
    k_irec_from_store<<<(m + 255) / 256, 256, 0, s>>>(js, out, m);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const g6x_jrec *d_rec, int n, JStore js, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    pin_carveout(k_scatter);
    k_scatter<<<(n + 127) / 128, 128, 0, s>>>(d_rec, n, js);
    return cudaGetLastError();
}

cudaError_t launch_predict(int kind, JStore js, Pred p, int nj, int nj_pad,
                           double t, int sm_count, cudaStream_t s)
{
    return launch_update_predict(kind, js, p, nj, nj_pad, t, nullptr, nullptr, 0, sm_count, s);
}

cudaError_t launch_update_predict(int kind, JStore js, Pred p, int nj, int nj_pad, double t,
                                  const g6x_jrec *rec, const int *toff, int ntiles_all,
                                  int sm_count, cudaStream_t s)
{
    const bool upd = rec != nullptr && toff != nullptr && ntiles_all > 0;
    const int nt = upd ? ntiles_all : nj_pad / JT;
    int blocks = nt;
    const int cap = sm_count * 8;
    if (blocks > cap)
        blocks = cap;
    if (blocks < 1)
        blocks = 1;
#define G6_K1(K, U)                                                                       \
    do {                                                                                  \
        pin_carveout(k_predict<K, U>);                                                    \
        k_predict<K, U><<<blocks, JT, 0, s>>>(js, p, nj, nj_pad, t, rec, toff, ntiles_all); \
    } while (0)
    if (kind == PRED_FP64) {
        if (upd) G6_K1(PRED_FP64, true); else G6_K1(PRED_FP64, false);
    } else if (kind == PRED_DS_X64) {
        if (upd) G6_K1(PRED_DS_X64, true); else G6_K1(PRED_DS_X64, false);
    } else {
        if (upd) G6_K1(PRED_DS, true); else G6_K1(PRED_DS, false);
    }
#undef G6_K1
    return cudaGetLastError();
}

// Arguments of the fused prediction (variants with fpred set).
static bool set_fused_pred(ForceArgs &a, const ForceConfig &cfg, const FusedPred *fp)
{
    if (cfg.ws || cfg.variant < 0 || cfg.variant >= kNumVariants)
        return false;
    if (!kVariants[cfg.variant].info.fpred)
        return true;
    if (!fp)
        return false;
    a.js = fp->js;
    a.t_pred = fp->t;
    a.nj = fp->nj;
    a.rec = fp->rec;
    a.toff = fp->toff;
    return fp->rec == nullptr || (cfg.n_itile == 1 && fp->toff != nullptr);
}


cudaError_t launch_force(const ForceConfig &cfg, const Pred &p,
                         const g6x_irec *d_irec, int ni, double eps2,
                         void *part, int *nbl_part, int *nbc_part,
                         int *d_err, cudaStream_t s, const FusedPred *fp, bool pdl,
                         const ListArgs *lists)
{
    if (cfg.work <= 0)
        return cudaSuccess;
    if (cfg.ws || cfg.variant < 0 || cfg.variant >= kNumVariants)
        return cudaErrorInvalidValue;           // small-block kernel: launch_force_ws
    cudaError_t e = prepare_variant(cfg.variant);
    if (e != cudaSuccess)
        return e;
    ForceArgs a{};
    a.pt = p.pt;
    a.trange = p.trange;
    a.p64 = p.p64;
    a.v64 = p.v64;
    a.irec = d_irec;
    a.part = part;
    a.nbl = nbl_part;
    a.nbc = nbc_part;
    if (lists) {
        a.maxnb = lists->maxnb;
        a.nbseg = lists->nbseg;
        a.nbmax = lists->nbmax;
    }
    if (cfg.list && (!lists || !lists->nbmax || lists->nbseg < 1 || lists->nbseg > lists->maxnb))
        return cudaErrorInvalidValue;
    if (cfg.list && cfg.tj > 1)
        a.nbr = nbl_part + partial_slots(cfg) * (size_t)lists->nbseg;
    a.err = d_err;
    a.W = cfg.work;
    a.J = cfg.jtiles;
    a.ni = ni;
    a.eps2 = eps2;
    a.wait_ns = g_wait_ns;
    if (!set_fused_pred(a, cfg, fp))
        return cudaErrorInvalidValue;
    const Variant &v = kVariants[cfg.variant];
    return launch_maybe_pdl(v.fn, cfg.grid, v.threads, v.smem, s, pdl, a);
}

cudaError_t launch_force_fused(const ForceConfig &cfg, const Pred &p,
                               const g6x_irec *d_irec, int ni, double eps2, void *part,
                               int *d_err, g6x_out *out, const int *jidx, unsigned *tcnt,
                               cudaStream_t s, const FusedPred *fp, bool pdl,
                               const ListArgs *lists)
{
    if (cfg.work <= 0)
        return cudaSuccess;
    if (cfg.prec != G6X_PREC_DS || cfg.ws || cfg.variant < 0 || cfg.variant >= kNumVariants)
        return cudaErrorInvalidValue;
    if (cfg.list
        && (!lists || !lists->nbmax || lists->nbseg < 1 || lists->nbseg > lists->maxnb
            || !lists->nbl_part || !lists->nbc_part || !lists->nbl_out || !lists->nblen_out))
        return cudaErrorInvalidValue;
    cudaError_t e = prepare_variant(cfg.variant);
    if (e != cudaSuccess)
        return e;
    ForceArgs a{};
    a.pt = p.pt;
    a.trange = p.trange;
    a.p64 = p.p64;
    a.v64 = p.v64;
    a.irec = d_irec;
    a.part = part;
    a.err = d_err;
    a.W = cfg.work;
    a.J = cfg.jtiles;
    a.ni = ni;
    a.eps2 = eps2;
    a.out = out;
    a.jidx = jidx;
    a.tcnt = tcnt;
    a.fused = 1;
    a.wait_ns = g_wait_ns;
    if (cfg.list) {
        a.maxnb = lists->maxnb;
        a.nbseg = lists->nbseg;
        a.nbmax = lists->nbmax;
        a.nbl = lists->nbl_part;
        a.nbc = lists->nbc_part;
        a.nbl_out = lists->nbl_out;
        a.nblen_out = lists->nblen_out;
        if (cfg.tj > 1)
            a.nbr = lists->nbl_part + partial_slots(cfg) * (size_t)lists->nbseg;
    }
    if (!set_fused_pred(a, cfg, fp))
        return cudaErrorInvalidValue;
    const Variant &v = kVariants[cfg.variant];
    return launch_maybe_pdl(v.fn, cfg.grid, v.threads, v.smem, s, pdl, a);
}

cudaError_t launch_reduce(const ForceConfig &cfg, const void *part,
                          const int *nbl_part, const int *nbc_part,
                          const int *jidx, int ni, g6x_out *d_out, int *d_nbl,
                          int *d_nblen, cudaStream_t s, bool pdl, const ListArgs *lists)
{
    if (ni <= 0)
        return cudaSuccess;
    if (cfg.ws)
        return cudaErrorInvalidValue;           // the small-block kernel reduces itself
    ReduceArgs a;
    a.part = part;
    a.nbl = nbl_part;
    a.nbc = nbc_part;
    a.jidx = jidx;
    a.out = d_out;
    a.nbl_out = d_nbl;
    a.nblen_out = d_nblen;
    a.W = cfg.work;
    a.J = cfg.jtiles;
    a.G = cfg.grid;
    a.ni = ni;
    a.itile = cfg.itile;
    a.list = cfg.list;
    a.maxnb = lists ? lists->maxnb : 0;
    a.nbseg = lists ? lists->nbseg : 0;
    a.fused = 0;
    if (cfg.list && !lists)
        return cudaErrorInvalidValue;
    // many partials per i-particle (small blocks spread over many CTAs):
    // one CTA per i-particle; otherwise one warp per i-particle
    const long long per_i = (long long)cfg.grid / cfg.n_itile + 1;
    const bool wide = per_i >= 64;
    const int blocks = wide ? ni : (int)(((long long)ni * 32 + 255) / 256);
    if (cfg.prec == G6X_PREC_FP64) {
        if (wide) {
            pin_carveout(k_reduce_wide<Partial64>);
            return launch_maybe_pdl(k_reduce_wide<Partial64>, blocks, 256, 0, s, pdl, a);
        }
        pin_carveout(k_reduce<Partial64>);
        return launch_maybe_pdl(k_reduce<Partial64>, blocks, 256, 0, s, pdl, a);
    }
    if (wide) {
        pin_carveout(k_reduce_wide<PartialDS>);
        return launch_maybe_pdl(k_reduce_wide<PartialDS>, blocks, 256, 0, s, pdl, a);
    }
    pin_carveout(k_reduce<PartialDS>);
    return launch_maybe_pdl(k_reduce<PartialDS>, blocks, 256, 0, s, pdl, a);
}

// ---------------------------------------------------------------- batch ---

int batch_variant_count() { return kNumBatchVariants; }

VariantInfo batch_variant_info(int v) { return kBatchVariants[v].info; }

int batch_variant_occupancy(int v)
{
    if (v < 0 || v >= kNumBatchVariants)
        return 0;
    if (g_bocc[v] == 0) {
        const Variant &bv = kBatchVariants[v];
        if (cudaFuncSetAttribute(bv.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bv.smem)
            != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaFuncSetAttribute(reinterpret_cast<const void *>(bv.fn),
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bv.fn, bv.threads, bv.smem)
            != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        g_bocc[v] = n;
    }
    return g_bocc[v];
}

cudaError_t launch_predict_batch(int kind, JStore js, Pred p, BatchPredTables bp,
                                 const g6x_jrec *rec, const int *toff, int tile0, int ntiles,
                                 int sm_count, cudaStream_t s)
{
    if (ntiles <= 0)
        return cudaSuccess;
    int blocks = ntiles < sm_count * 8 ? ntiles : sm_count * 8;
#define G6_KB(K)                                                                        \
    do {                                                                                \
        pin_carveout(k_predict_batch<K>);                                               \
        k_predict_batch<K><<<blocks, JT, 0, s>>>(js, p, bp, rec, toff, tile0, ntiles); \
    } while (0)
    if (kind == PRED_FP64)
        G6_KB(PRED_FP64);
    else if (kind == PRED_DS_X64)
        G6_KB(PRED_DS_X64);
    else
        G6_KB(PRED_DS);
#undef G6_KB
    return cudaGetLastError();
}

cudaError_t launch_force_batch(int v, int grid, const Pred &p, const g6x_irec *d_irec,
                               void *part, int *d_err, const BatchTables &bt, cudaStream_t s,
                               unsigned *tcnt, g6x_out *out, const int *jidx)
{
    if (v < 0 || v >= kNumBatchVariants || grid < 1)
        return cudaErrorInvalidValue;
    if (batch_variant_occupancy(v) < 1)
        return cudaErrorInvalidConfiguration;
    ForceArgs a{};
    a.pt = p.pt;
    a.trange = p.trange;
    a.irec = d_irec;
    a.part = part;
    a.err = d_err;
    a.bt = bt;
    a.wait_ns = g_wait_ns;
    if (tcnt) {
        a.fused = 1;
        a.tcnt = tcnt;
        a.out = out;
        a.jidx = jidx;
    }
    const Variant &bv = kBatchVariants[v];
    bv.fn<<<grid, bv.threads, bv.smem, s>>>(a);
    return cudaGetLastError();
}

void set_wait_limit_ns(unsigned long long ns) { g_wait_ns = ns; }

unsigned long long wait_limit_ns() { return g_wait_ns; }

unsigned long long max_wait_limit_ns() { return WAIT_LIMIT_NS; }

cudaError_t launch_wait_probe(int *d_err, cudaStream_t s)
{
    k_wait_probe<<<1, 32, 0, s>>>(d_err, g_wait_ns);
    return cudaGetLastError();
}

cudaError_t launch_reduce_batch(int v, int grid, const void *part, const int *jidx,
                                g6x_out *d_out, const BatchTables &bt, int blocks,
                                cudaStream_t s, bool fused)
{
    if (v < 0 || v >= kNumBatchVariants)
        return cudaErrorInvalidValue;
    ReduceArgs a{};
    a.part = part;
    a.jidx = jidx;
    a.out = d_out;
    a.G = grid;
    a.itile = kBatchVariants[v].info.ti * kBatchVariants[v].info.nper;
    a.fused = fused ? 1 : 0;
    pin_carveout(k_reduce_batch<PartialDS>);
    k_reduce_batch<PartialDS><<<blocks, 256, 0, s>>>(a, bt);
    return cudaGetLastError();
}

}  // namespace g6
