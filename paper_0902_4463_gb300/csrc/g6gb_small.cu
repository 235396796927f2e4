// g6gb_small.cu -- K2s, the force kernel for small active blocks
// (Gaburov, Harfst & Portegies Zwart, arXiv:0902.4463, Sect. 2.1 and 2.3).
//
// In a block-time-step run most block steps move a few particles, and each
// of them still needs every j-particle predicted to the block time (Eq. 1,
// Eq. 2) and summed over (Sect. 2.1: the force is O(nm), the prediction
// O(n)).  With m i-particles and n j-particles the step is then bound by the
// stream of n raw j-records (84 B each) and by latency, not by the pair
// arithmetic.  This kernel serves blocks of up to 256 i-particles in one
// launch:
//
//   * the whole block is one i-tile held by every CTA; the j-tiles are split
//     evenly over the CTAs (the paper's j split over the multiprocessors, and
//     its extra split of j inside a block for small m, Sect. 2.3);
//   * warp specialisation: one producer warp streams the CTA's raw j-tiles
//     (t0, v, a/2, j/6, DS position, index) into a ring of SR shared-memory
//     stages with bulk asynchronous copies; the compute warps predict each
//     tile into one of two predicted-tile buffers (the K1 arithmetic, so the
//     tiles are bit-identical to K1's), one tile ahead of the pair loop that
//     reads the other buffer.  The raw stages pass between the producer and
//     the compute warps on mbarriers, so the copies of later tiles stay in
//     flight while the compute warps work; the compute warps alone meet at
//     one named barrier per tile, which releases both predicted buffers;
//   * the staged j-records of the CTA's own tiles (the j-store update of
//     Sect. 2.1) are stored by the producer warp before its first copy;
//   * the partial sums of the CTAs are reduced inside the launch in two
//     levels: the last CTA of each group of gs CTAs sums the group's partials,
//     the last group to finish sums the group results and writes the forces
//     (Sect. 2.3: the partial forces are reduced on the GPU).  The summation
//     order is fixed by CTA and group index, so results do not depend on which
//     CTA finishes last.
//
// The pair arithmetic and the compensated accumulation are those of K2
// (k_force_ds); the nearest neighbour is found from the tile still in
// shared memory whenever a tile lowers a thread's smallest key, instead of
// K2's rescan of the winning tile from global memory at the end.  Every wait
// is bounded; a wait that runs out records G6_ETIMEDOUT in the error word and
// makes the other warps give up at their next wait, and the producer warp
// keeps the CTA alive until every copy it issued has landed.
#include "g6gb_device.cuh"

#include <climits>
#include <cmath>
#include <type_traits>

namespace g6 {

namespace {

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(bar)) : "memory");
}

// Bounded wait of one thread for phase `parity`: false when the limit ran
// out (then G6_ETIMEDOUT is recorded and the abort flag raised) or another
// warp has given up.
__device__ __forceinline__ bool ws_wait1(uint64_t *bar, uint32_t parity,
                                         unsigned long long limit, volatile int *abort_flag,
                                         int *err)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 8; ++k)
            if (mbar_try_wait(bar, parity))
                return true;
        if (*abort_flag)
            return false;
        if (global_ns() - t0 > limit) {
            *abort_flag = 1;
            *(volatile int *)err = G6_ETIMEDOUT;
            return false;
        }
    }
}

// The same for a whole warp: lane 0 waits, the warp takes its answer, and
// after a completed phase every lane observes it once more (that phase
// cannot be overtaken before this warp has arrived on its partner barrier)
// so that each lane acquires what the phase released.
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, unsigned long long limit,
                                        volatile int *abort_flag, int *err)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0)
        ok = ws_wait1(bar, parity, limit, abort_flag, err);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (ok)
        mbar_try_wait(bar, parity);
    return ok;
}

// One partial record read past L1 (written by other CTAs of this launch).
__device__ __forceinline__ PartialDS load_partial_cg(const PartialDS *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 v0 = __ldcg(q), v1 = __ldcg(q + 1), v2 = __ldcg(q + 2), v3 = __ldcg(q + 3);
    PartialDS r;
    r.acc[0] = make_float2(v0.x, v0.y);
    r.acc[1] = make_float2(v0.z, v0.w);
    r.acc[2] = make_float2(v1.x, v1.y);
    r.jerk[0] = make_float2(v1.z, v1.w);
    r.jerk[1] = make_float2(v2.x, v2.y);
    r.jerk[2] = make_float2(v2.z, v2.w);
    r.pot = make_float2(v3.x, v3.y);
    r.nnr2 = v3.z;
    r.nnj = __float_as_int(v3.w);
    return r;
}

static_assert(sizeof(PartialDS) == 64, "partial record is four float4");

}  // namespace

// TI threads along i x TJ j-groups = 256 compute threads (8 warps, one
// j-particle each when a tile is predicted), NI i-particles per thread, so
// the i-tile is TI x NI; one producer warp; MINB CTAs per SM; SR raw stages;
// UNR j-pairs of the pair loop unrolled together.
template <int TI, int TJ, int NI, int MINB, int SR, int UNR = 2>
__global__ void __launch_bounds__(TI * TJ + 32, MINB) k_force_ws(const ForceArgs a)
{
    constexpr int NT = TI * TJ;                       // compute threads
    constexpr int NW = NT / 32;                       // compute warps
    constexpr int ITILE = TI * NI;
    constexpr int PPT = JT / 2 / TJ;                  // j-pairs per thread per tile
    constexpr int FLUSH = (256 + PPT - 1) / PPT;      // tiles between flushes (>= 512 j)
    constexpr int CHP = PPT < 4 ? PPT : 4;            // j-pairs per neighbour-search chunk
    static_assert(PPT % CHP == 0, "whole chunks per tile");
    constexpr int PT_WORDS = JW * JT;                 // one predicted tile
    static_assert(NT == JT, "one j-particle per compute thread when a tile is predicted");
    static_assert(JT % (2 * TJ) == 0, "j-tile must split into j-pairs evenly");
    // nothing is read before the predecessor (a j-store update) has completed
    grid_dep_wait();
    grid_dep_launch();

    extern __shared__ __align__(128) unsigned char dyn_smem[];
    unsigned char *raw = dyn_smem;                                          // SR raw stages
    float *pbuf = reinterpret_cast<float *>(dyn_smem + SR * RAW_TILE_BYTES);  // 2 predicted tiles
    float2 *comp = reinterpret_cast<float2 *>(dyn_smem + SR * RAW_TILE_BYTES
                                              + 2 * PT_WORDS * sizeof(float));   // [NI][7][NT]
    __shared__ __align__(8) uint64_t rfull[SR], rempty[SR];
    __shared__ int2 s_wr[2][NW];                      // per predicted tile: each warp's index range
    __shared__ int s_abort, s_last1, s_last2;
    __shared__ float s_ibuf[TJ > 1 ? 11 * ITILE : 1];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, c = blockIdx.x;
    const int jb = (int)((long long)c * a.J / G);
    const int ntile = (int)((long long)(c + 1) * a.J / G) - jb;
    volatile int *abort_flag = &s_abort;

    // The producer warp sets up the barriers and, once the staged j-records
    // of its tiles are stored, issues the first SR copies; meanwhile the
    // compute warps split the i-positions.  One CTA barrier then makes the
    // barriers and the i-data visible to everyone; after it every wait is an
    // mbarrier wait with a limit.
    int issued = 0;                                   // producer lane 0: tiles issued
    auto issue = [&](int q) {
        const int s = q % SR;
        mbar_expect_tx(&rfull[s], RAW_TILE_BYTES);
        bulk_g2s(raw + (size_t)s * RAW_TILE_BYTES, raw_tile(a.js, jb + q), RAW_TILE_BYTES,
                 &rfull[s]);
    };
    if (warp == NW) {
        // the staged j-records of this CTA's tiles (sorted by tile, so one
        // contiguous range), stored before any copy reads the tiles
        if (a.rec && ntile > 0) {
            const int r0 = a.toff[jb], r1 = a.toff[jb + ntile];
            for (int r = r0 + lane; r < r1; r += 32)
                store_record(a.rec[r], a.js);
            fence_proxy_async_global();
            __syncwarp();
        }
        if (lane == 0) {
            for (int s = 0; s < SR; ++s) {
                mbar_init(&rfull[s], 1);
                mbar_init(&rempty[s], NW);
            }
            fence_barrier_init();
            s_abort = 0;
            for (; issued < SR && issued < ntile; ++issued)
                issue(issued);
        }
    } else {
        if constexpr (TJ > 1) {
            // the DS split of the i-positions, once per i-particle
            for (int il = tid; il < ITILE; il += NT) {
                float w[11];
                if (il < a.ni) {
                    const g6x_irec &r = a.irec[il];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const double x = r.x[d];
                        const float hi = __double2float_rn(x);
                        w[d] = hi;
                        w[3 + d] = __double2float_rn(x - (double)hi);
                        w[6 + d] = (float)r.v[d];
                    }
                    w[9] = (float)r.h2;
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
        }
    }
    __syncthreads();

    // ------------------------------------------------------- producer warp
    if (warp == NW) {
        if (lane == 0) {
            int q = issued;
            for (; q < ntile; ++q) {
                const int s = q % SR;
                if (!ws_wait1(&rempty[s], (uint32_t)((q / SR - 1) & 1), a.wait_ns, abort_flag,
                              a.err))
                    break;
                issue(q);
            }
            // no copy may land in shared memory after the CTA has exited:
            // wait (always the full limit) for the last copy of every stage
            for (int r = q > SR ? q - SR : 0; r < q; ++r)
                mbar_wait_bounded(&rfull[r % SR], (uint32_t)((r / SR) & 1), WAIT_LIMIT_NS);
        }
        return;
    }

    // -------------------------------------------------------- compute warps
    // The compute warps meet at one named barrier per tile (the producer warp
    // is not part of it).  A warp that gives up at a bounded wait still
    // passes every barrier, skipping its work, so no warp can be left waiting
    // at one; the outcome is read once after the tile loop.
    auto cta_bar = [&]() { asm volatile("bar.sync 1, %0;" :: "n"(NT) : "memory"); };
    const int ti = tid % TI, tj = tid / TI;
    const float2 eps2 = make_float2((float)a.eps2, (float)a.eps2);
    const float2 m3 = make_float2(-3.0f, -3.0f);
    const float INF = __int_as_float(0x7f800000);
    float2 nxh[NI][3], nxl[NI][3], nv[NI][3];
    int iid[NI];
    float2 ta[NI][7];
    float tmin[NI], nnr[NI];
    int nnj[NI], tchk[NI];
    auto cslot = [&](int k, int q) -> float2 & { return comp[(k * 7 + q) * NT + tid]; };
#pragma unroll
    for (int k = 0; k < NI; ++k) {
        const int il = k * TI + ti;
        if constexpr (TJ > 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float hi = s_ibuf[d * ITILE + il], lo = s_ibuf[(3 + d) * ITILE + il];
                const float w = -s_ibuf[(6 + d) * ITILE + il];
                nxh[k][d] = make_float2(-hi, -hi);
                nxl[k][d] = make_float2(-lo, -lo);
                nv[k][d] = make_float2(w, w);
            }
            iid[k] = __float_as_int(s_ibuf[10 * ITILE + il]);
        } else if (il < a.ni) {
            const g6x_irec &r = a.irec[il];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double x = r.x[d];
                const float hi = __double2float_rn(x);
                const float lo = __double2float_rn(x - (double)hi);
                nxh[k][d] = make_float2(-hi, -hi);
                nxl[k][d] = make_float2(-lo, -lo);
                const float w = -(float)r.v[d];
                nv[k][d] = make_float2(w, w);
            }
            iid[k] = r.index;
        } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                nxh[k][d] = make_float2(0.f, 0.f);
                nxl[k][d] = make_float2(0.f, 0.f);
                nv[k][d] = make_float2(0.f, 0.f);
            }
            iid[k] = -2;
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            ta[k][q] = make_float2(0.f, 0.f);
            cslot(k, q) = make_float2(0.f, 0.f);
        }
        tmin[k] = INF;
        nnr[k] = INF;
        nnj[k] = -1;
        tchk[k] = 0;
    }

    // Eq. 1 and Eq. 2 for tile q (raw stage q % SR) into predicted buffer
    // q & 1, one j-particle per thread; each warp records its index range
    // and hands the raw stage back to the producer.
    auto predict_into = [&](int q) -> bool {
        const int r = q % SR, p = q & 1;
        if (!ws_wait(&rfull[r], (uint32_t)((q / SR) & 1), a.wait_ns, abort_flag, a.err))
            return false;
        const unsigned char *d = raw + (size_t)r * RAW_TILE_BYTES;
        const int jj = tid;
        const int slot = (jb + q) * JT + jj;
        float *o = pbuf + p * PT_WORDS + jj;
        int lo = INT_MAX, hi = -1;
        if (slot < a.nj) {
            const int id = reinterpret_cast<const int *>(d + RAW_ID)[jj];
            predict_ds_vals((float)(a.t_pred - reinterpret_cast<const double *>(d + RAW_T0)[jj]),
                            reinterpret_cast<const float4 *>(d + RAW_XA)[jj],
                            reinterpret_cast<const float2 *>(d + RAW_XB)[jj],
                            reinterpret_cast<const float4 *>(d + RAW_V)[jj],
                            reinterpret_cast<const float4 *>(d + RAW_A)[jj],
                            reinterpret_cast<const float4 *>(d + RAW_J)[jj], id, o);
            if (id >= 0) {
                lo = id;
                hi = id;
            }
        } else {
            far_slot_ds(o);
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0)
            s_wr[p][warp] = make_int2(lo, hi);
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&rempty[r]);
        return true;
    };

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

    // The key (softened |r|^2, +inf for the i-particle's own j) of j-pair jp
    // of a predicted tile, with the pair loop's own packed operations.
    auto pair_key = [&](const float *S, int jp, int k) -> float2 {
        const float2 xh = reinterpret_cast<const float2 *>(S + W_XH * JT)[jp];
        const float2 yh = reinterpret_cast<const float2 *>(S + W_YH * JT)[jp];
        const float2 zh = reinterpret_cast<const float2 *>(S + W_ZH * JT)[jp];
        const float2 xl = reinterpret_cast<const float2 *>(S + W_XL * JT)[jp];
        const float2 yl = reinterpret_cast<const float2 *>(S + W_YL * JT)[jp];
        const float2 zl = reinterpret_cast<const float2 *>(S + W_ZL * JT)[jp];
        const int2 id = reinterpret_cast<const int2 *>(S + W_ID * JT)[jp];
        const float2 dx = __fadd2_rn(__fadd2_rn(xh, nxh[k][0]), __fadd2_rn(xl, nxl[k][0]));
        const float2 dy = __fadd2_rn(__fadd2_rn(yh, nxh[k][1]), __fadd2_rn(yl, nxl[k][1]));
        const float2 dz = __fadd2_rn(__fadd2_rn(zh, nxh[k][2]), __fadd2_rn(zl, nxl[k][2]));
        float2 key = soft_r2(dx, dy, dz, eps2);
        key.x = (id.x == iid[k]) ? INF : key.x;
        key.y = (id.y == iid[k]) ? INF : key.y;
        return key;
    };

    // All pairs of the thread's share of one predicted tile (the K2 pair
    // arithmetic, Eq. 3 separations); SELF: with the per-pair self test.
    auto tile_pass = [&](const float *S, auto self_tag) {
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
                const float2 dx = __fadd2_rn(__fadd2_rn(xh, nxh[k][0]), __fadd2_rn(xl, nxl[k][0]));
                const float2 dy = __fadd2_rn(__fadd2_rn(yh, nxh[k][1]), __fadd2_rn(yl, nxl[k][1]));
                const float2 dz = __fadd2_rn(__fadd2_rn(zh, nxh[k][2]), __fadd2_rn(zl, nxl[k][2]));
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
        // by chunks of CHP j-pairs, noting the first chunk that reaches the
        // tile's minimum, so the neighbour search reads one chunk
        for (int ch = 0; ch < PPT / CHP; ++ch) {
            float cm[NI];
#pragma unroll
            for (int k = 0; k < NI; ++k)
                cm[k] = INF;
#pragma unroll UNR
            for (int u = 0; u < CHP; ++u)
                jpair(ch * CHP + u, cm);
#pragma unroll
            for (int k = 0; k < NI; ++k)
                if (cm[k] < tmin[k]) {
                    tmin[k] = cm[k];
                    tchk[k] = ch;
                }
        }
    };

    // ------------------------------------------------------------ j-tiles
    // Tile q+1 is predicted while tile q's pairs run, into the other buffer;
    // one barrier per tile then releases both buffers.  Where a tile lowers
    // an i-particle's smallest key, the first j of the thread's share with
    // that key is found at once from the tile still in shared memory, in the
    // chunk the pair loop noted (ties to the lower j-slot: tiles, chunks and
    // shares are walked in ascending j).
    bool ok = ntile <= 0 || predict_into(0);
    cta_bar();
    int since_flush = 0;
    for (int q = 0; q < ntile; ++q) {
        ok = ok && !*abort_flag;
        if (ok && q + 1 < ntile)
            ok = predict_into(q + 1);
        const int p = q & 1;
        if (ok) {
            int2 rg = make_int2(INT_MAX, -1);
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int2 v = s_wr[p][w];
                rg.x = min(rg.x, v.x);
                rg.y = max(rg.y, v.y);
            }
            bool mine = false;
#pragma unroll
            for (int k = 0; k < NI; ++k)
                mine |= (iid[k] >= rg.x && iid[k] <= rg.y);
            const float *S = pbuf + p * PT_WORDS;
            if (__any_sync(0xffffffffu, mine))
                tile_pass(S, std::true_type{});
            else
                tile_pass(S, std::false_type{});
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                if (tmin[k] < nnr[k]) {
                    nnr[k] = tmin[k];
                    for (int kk = tchk[k] * CHP; kk < (tchk[k] + 1) * CHP; ++kk) {
                        const float2 key = pair_key(S, tj + kk * TJ, k);
                        if (key.x == nnr[k] || key.y == nnr[k]) {
                            nnj[k] = (jb + q) * JT + 2 * (tj + kk * TJ) + (key.x == nnr[k] ? 0 : 1);
                            break;
                        }
                    }
                }
                tmin[k] = INF;
            }
            if (++since_flush >= FLUSH) {
                flush();
                since_flush = 0;
            }
        }
        cta_bar();
    }
    // one reading of the outcome for all compute warps
    if (tid == 0)
        s_last1 = *abort_flag;
    cta_bar();
    if (s_last1)
        return;

    // ------------------------------------------------------------ epilogue
    flush();
    PartialDS *P0 = static_cast<PartialDS *>(a.part);  // [G][ITILE], this CTA's sums
    if constexpr (TJ > 1) {
        // The TJ j-groups of an i-particle combine in compensated FP32,
        // nearest neighbour ties to the lower j-slot.  First inside each warp:
        // with TI < 32 a warp holds 32 / TI groups of the same TI particles,
        // combined by shuffles over the lane bits above TI.  Then the NH
        // holders of each i-particle (one per warp, or one per warp with the
        // same i-range when TI >= 32) meet in the raw stages, free now that
        // every copy has landed and been read, in a fixed holder order.
        constexpr int TIW = TI < 32 ? TI : 32;        // particles of a warp's holders
        constexpr int WPI = TI / TIW;                 // warps across one i-range
        constexpr int NH = NW / WPI;                  // holders per i-particle
        float2 *hsum = reinterpret_cast<float2 *>(raw);                        // [NH][NI][7][TI]
        float *hnr = reinterpret_cast<float *>(hsum + NH * NI * 7 * TI);       // [NH][NI][TI]
        int *hnj = reinterpret_cast<int *>(hnr + NH * NI * TI);                // [NH][NI][TI]
        static_assert((NH * NI * 7 * TI * 8 + 2 * NH * NI * TI * 4) <= (int)RAW_TILE_BYTES * SR,
                      "holder sums fit the raw stages");
        const int hidx = warp / WPI, hti = (warp % WPI) * TIW + lane;
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            float h[7], l[7];
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const float2 hl = cslot(k, q);
                h[q] = hl.x;
                l[q] = hl.y;
            }
            float br = nnr[k];
            int bj = nnj[k];
#pragma unroll
            for (int off = TIW; off < 32; off <<= 1) {
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const float oh = __shfl_xor_sync(0xffffffffu, h[q], off);
                    const float ol = __shfl_xor_sync(0xffffffffu, l[q], off);
                    ds_acc(h[q], l[q], oh, ol);
                }
                const float r = __shfl_xor_sync(0xffffffffu, br, off);
                const int jj = __shfl_xor_sync(0xffffffffu, bj, off);
                if (jj >= 0 && (bj < 0 || r < br || (r == br && jj < bj))) {
                    br = r;
                    bj = jj;
                }
            }
            if (lane < TIW) {
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    hsum[((hidx * NI + k) * 7 + q) * TI + hti] = make_float2(h[q], l[q]);
                hnr[(hidx * NI + k) * TI + hti] = br;
                hnj[(hidx * NI + k) * TI + hti] = bj;
            }
        }
        cta_bar();
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
            for (int g = 0; g < NH; ++g) {
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    const float2 hl = hsum[((g * NI + k) * 7 + q) * TI + ii];
                    ds_acc(sh[q], sl[q], hl.x, hl.y);
                }
                const float r = hnr[(g * NI + k) * TI + ii];
                const int jj = hnj[(g * NI + k) * TI + ii];
                if (jj >= 0 && (r < br || (r == br && (bj < 0 || jj < bj)))) {
                    br = r;
                    bj = jj;
                }
            }
            PartialDS *P = P0 + (size_t)c * ITILE + il;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                P->acc[d] = make_float2(sh[d], sl[d]);
                P->jerk[d] = make_float2(sh[3 + d], sl[3 + d]);
            }
            P->pot = make_float2(sh[6], sl[6]);
            P->nnr2 = unsoftened(br, eps2.x);
            P->nnj = bj;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            PartialDS *P = P0 + (size_t)c * ITILE + k * TI + ti;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                P->acc[d] = cslot(k, d);
                P->jerk[d] = cslot(k, 3 + d);
            }
            P->pot = cslot(k, 6);
            P->nnr2 = unsoftened(nnr[k], eps2.x);
            P->nnj = nnj[k];
        }
    }

    // Sum of nrec partial records src[q * ITILE + il] per i-particle, in
    // record order: P lanes per i-particle (a power of two) take records
    // q = lane, lane + P, ... and combine by shuffles.  Writes a partial
    // record to dst, or with dst == nullptr the forces of the block.
    auto reduce_records = [&](const PartialDS *src, int nrec, PartialDS *dst) {
        int P = 1;
        while (P < 32 && 2 * P <= nrec && 2 * P * ITILE <= NT)
            P *= 2;
        const int groups = NT / P;
        const int rounds = (ITILE + groups - 1) / groups;
        const int part = tid % P;
        for (int rr = 0; rr < rounds; ++rr) {
            const int il = rr * groups + tid / P;
            PartialSum<PartialDS> acc;
            acc.init();
            if (il < ITILE) {
#pragma unroll 4
                for (int q = part; q < nrec; q += P)
                    acc.add(load_partial_cg(src + (size_t)q * ITILE + il));
            }
            for (int off = P / 2; off > 0; off >>= 1)
                acc.shfl_combine(off);
            if (il < ITILE && part == 0) {
                if (dst) {
                    PartialDS *D = dst + il;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        D->acc[d] = make_float2(acc.h[d], acc.l[d]);
                        D->jerk[d] = make_float2(acc.h[3 + d], acc.l[3 + d]);
                    }
                    D->pot = make_float2(acc.h[6], acc.l[6]);
                    D->nnr2 = acc.br;
                    D->nnj = acc.bj;
                } else if (il < a.ni) {
                    a.out[il] = result_of(acc, a.jidx);
                }
            }
        }
    };

    // Two-level reduction: the last CTA of each group of gs CTAs sums the
    // group, the last group sums the groups.  Each counter is reset by the
    // CTA that completes it, so it is zero again after a complete launch.
    __threadfence();
    cta_bar();
    const int gs = a.gs;
    const int NG = (G + gs - 1) / gs;
    const int g = c / gs, g0 = g * gs;
    const int gn = min(G, g0 + gs) - g0;
    if (tid == 0)
        s_last1 = atomicAdd(&a.tcnt[g], 1u) + 1 == (unsigned)gn;
    cta_bar();
    if (!s_last1)
        return;
    __threadfence();
    PartialDS *P1 = P0 + (size_t)G * ITILE;           // [NG][ITILE], group sums
    reduce_records(P0 + (size_t)g0 * ITILE, gn, NG > 1 ? P1 + (size_t)g * ITILE : nullptr);
    if (tid == 0)
        a.tcnt[g] = 0u;
    if (NG == 1)
        return;
    __threadfence();
    cta_bar();
    if (tid == 0)
        s_last2 = atomicAdd(&a.tcnt[NG], 1u) + 1 == (unsigned)NG;
    cta_bar();
    if (!s_last2)
        return;
    __threadfence();
    reduce_records(P1, NG, nullptr);
    if (tid == 0)
        a.tcnt[NG] = 0u;
}

// ------------------------------------------------------------ variants ---

namespace {

using WsFn = void (*)(const ForceArgs);

struct WsVariant {
    VariantInfo info;
    WsFn fn;
    int smem;
};

// dynamic shared memory: SR raw stages, two predicted tiles, the
// compensated sums of 256 compute threads
constexpr int ws_smem(int sr, int ni)
{
    return sr * (int)RAW_TILE_BYTES + 2 * JW * JT * (int)sizeof(float) + ni * 7 * 256 * 8;
}

// VariantInfo: ti, tj, nper, list, prec, fpred, twin, ws
const WsVariant kWs[] = {
    {{16, 16, 1, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<16, 16, 1, 2, 3>, ws_smem(3, 1)},
    {{32, 8, 1, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<32, 8, 1, 2, 3>, ws_smem(3, 1)},
    {{64, 4, 1, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<64, 4, 1, 2, 3>, ws_smem(3, 1)},
    {{128, 2, 1, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<128, 2, 1, 2, 3>, ws_smem(3, 1)},
    {{256, 1, 1, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<256, 1, 1, 2, 3>, ws_smem(3, 1)},
    // two i-particles per thread, one CTA per SM with a deeper ring
    {{16, 16, 2, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<16, 16, 2, 1, 6>, ws_smem(6, 2)},
    {{32, 8, 2, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<32, 8, 2, 1, 6>, ws_smem(6, 2)},
    {{64, 4, 2, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<64, 4, 2, 1, 6>, ws_smem(6, 2)},
    {{128, 2, 2, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<128, 2, 2, 1, 6>, ws_smem(6, 2)},
    // the narrowest i-tile, for blocks of up to 8
    {{8, 32, 1, 0, G6X_PREC_DS, 1, -1, 1}, k_force_ws<8, 32, 1, 2, 3>, ws_smem(3, 1)},
};
constexpr int kNumWs = (int)(sizeof(kWs) / sizeof(kWs[0]));
int g_ws_occ[kNumWs];

}  // namespace

int ws_variant_count() { return kNumWs; }

VariantInfo ws_variant_info(int k) { return kWs[k].info; }

int ws_variant_smem(int k) { return kWs[k].smem; }

int ws_variant_threads(int) { return JT + 32; }

int ws_variant_occupancy(int k)
{
    if (k < 0 || k >= kNumWs)
        return 0;
    if (g_ws_occ[k] == 0) {
        const WsVariant &v = kWs[k];
        if (cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem)
            != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaFuncSetAttribute(reinterpret_cast<const void *>(v.fn),
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaGetLastError();
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v.fn, JT + 32, v.smem)
            != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        g_ws_occ[k] = n;
    }
    return g_ws_occ[k];
}

int ws_group_size(int grid)
{
    int gs = 1;
    while (gs * gs < grid)
        ++gs;
    return gs;
}

size_t ws_partial_slots(int grid, int itile)
{
    const int gs = ws_group_size(grid);
    return (size_t)(grid + (grid + gs - 1) / gs) * itile;
}

cudaError_t launch_force_ws(const ForceConfig &cfg, const g6x_irec *d_irec, int ni, double eps2,
                            int nj, void *part, unsigned *cnt, g6x_out *out, const int *jidx,
                            int *d_err, const FusedPred &fp, cudaStream_t s, bool pdl)
{
    const int k = cfg.variant - (variant_count() - kNumWs);
    const int grid = cfg.grid, jtiles = cfg.jtiles;
    if (!cfg.ws || k < 0 || k >= kNumWs || grid < 1 || grid > jtiles || ni < 1
        || ni > kWs[k].info.ti * kWs[k].info.nper)
        return cudaErrorInvalidValue;
    if (ws_variant_occupancy(k) < 1)
        return cudaErrorInvalidConfiguration;
    ForceArgs a{};
    a.irec = d_irec;
    a.part = part;
    a.err = d_err;
    a.J = jtiles;
    a.ni = ni;
    a.eps2 = eps2;
    a.out = out;
    a.jidx = jidx;
    a.tcnt = cnt;
    a.fused = 1;
    a.wait_ns = wait_limit_ns();
    a.js = fp.js;
    a.t_pred = fp.t;
    a.nj = nj;
    a.rec = fp.rec;
    a.toff = fp.toff;
    a.gs = ws_group_size(grid);
    const WsVariant &v = kWs[k];
    return launch_maybe_pdl(v.fn, grid, JT + 32, v.smem, s, pdl, a);
}

}  // namespace g6
