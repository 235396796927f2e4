// g6gb_device.cuh -- device-side pieces shared by the force kernels of the
// direct-summation hot path (arXiv:0902.4463): mbarrier and bulk-copy
// primitives, compensated FP32 sums, the j-store record store (Sect. 2.1),
// the double-single predictor of Sect. 2.2, the force-kernel arguments and
// the partial-sum reduction of Sect. 2.3.  Included by the kernel sources
// only; not installed.
#pragma once

#include "g6gb_internal.h"

#include <climits>
#include <cuda_runtime.h>

namespace g6 {

namespace {

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s per mbarrier wait


__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x on the multi-function unit (the pair loops take r^-2 from here rather
// than as r^-1 * r^-1, one operation less on the FP32 pipe): +inf -> 0.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Softened |r|^2 = dx^2 + dy^2 + dz^2 + eps^2 of a j-pair (packed FP32x2),
// eps^2 folded into the first fused multiply-add.  The pair loops use it as
// the nearest-neighbour and list key (in exact arithmetic the same order as
// |r|^2, eps^2 being one constant per call); the rescans that find the
// winning j use the scalar form, whose lanes round identically.
__device__ __forceinline__ float2 soft_r2(float2 dx, float2 dy, float2 dz, float2 e2)
{
    return __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e2)));
}

__device__ __forceinline__ float soft_r2(float dx, float dy, float dz, float e2)
{
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, e2)));
}

// A partial record's nearest-neighbour distance without the softening
// (+inf stays +inf; rounding is monotone, so no two records change order).
__device__ __forceinline__ float unsoftened(float key, float e2)
{
    return fmaxf(__fsub_rn(key, e2), 0.f);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                 :: "r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier for at most limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 32; ++k)
            if (mbar_try_wait(bar, parity))
                return true;
        if (global_ns() - t0 > limit_ns)
            return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier global stores before later bulk asynchronous
// copies (the async proxy) that read them.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor in the stream still runs;
// grid_dep_wait() blocks until every prerequisite grid has completed and its
// memory operations are visible (a no-op without such a predecessor), and
// grid_dep_launch() lets the dependent grid be scheduled once every CTA of
// this grid has issued it or exited.
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (ah, al) += (bh, bl) in compensated FP32: TwoSum of the high parts, the
// low parts added to the error, renormalised (Fast2Sum).
__device__ __forceinline__ void ds_acc(float &ah, float &al, float bh, float bl)
{
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    ah = __fadd_rn(s, e);
    al = __fsub_rn(e, __fsub_rn(ah, s));
}

// Work line helpers: CTA c owns [begin(c), begin(c+1)).
__device__ __forceinline__ long long work_begin(long long c, long long W, long long G)
{
    return c * W / G;
}

// Largest c with work_begin(c) <= p, i.e. the CTA that owns position p.
__device__ __forceinline__ long long work_owner(long long p, long long W, long long G)
{
    return ((p + 1) * G - 1) / W;
}

// Whether the i-tile owned by CTAs clo .. chi is reduced by the last of them
// inside the force launch: few of them, and every one with work (a line
// shorter than the grid leaves CTAs without work, which never arrive).
__device__ __forceinline__ bool fused_span(long long clo, long long chi, long long W, long long G)
{
    if (chi - clo + 1 > FUSED_MAX_SEGS)
        return false;
    for (long long c = clo; c <= chi; ++c)
        if (work_begin(c, W, G) == work_begin(c + 1, W, G))
            return false;
    return true;
}

// Far-away massless stand-in for padding and empty j-slots: every pair term
// it produces is exactly zero (r^2 overflows to +inf, rsqrt(+inf) = 0).
constexpr double FAR = 1e30;

}  // namespace

// Entry of slot k in one plane of the tiled raw j-store.
template <class T>
__device__ __forceinline__ T &raw_at(const JStore &js, unsigned plane, int k)
{
    return *reinterpret_cast<T *>(js.raw + (size_t)(k / JT) * RAW_TILE_BYTES + plane
                                  + (size_t)(k % JT) * sizeof(T));
}
__device__ __forceinline__ double &js_t0(const JStore &js, int k) { return raw_at<double>(js, RAW_T0, k); }
__device__ __forceinline__ float4 &js_v0m(const JStore &js, int k) { return raw_at<float4>(js, RAW_V, k); }
__device__ __forceinline__ float4 &js_a2f(const JStore &js, int k) { return raw_at<float4>(js, RAW_A, k); }
__device__ __forceinline__ float4 &js_j6f(const JStore &js, int k) { return raw_at<float4>(js, RAW_J, k); }
__device__ __forceinline__ float4 &js_xds(const JStore &js, int k) { return raw_at<float4>(js, RAW_XA, k); }
__device__ __forceinline__ float2 &js_xds2(const JStore &js, int k) { return raw_at<float2>(js, RAW_XB, k); }
__device__ __forceinline__ int &js_idx(const JStore &js, int k) { return raw_at<int>(js, RAW_ID, k); }
__device__ __forceinline__ const unsigned char *raw_tile(const JStore &js, int tile)
{
    return js.raw + (size_t)tile * RAW_TILE_BYTES;
}

// Store one j-particle record in its j-memory slot (the j-store update of
// Sect. 2.1: only corrected particles travel to the GPU each step).
__device__ __forceinline__ void store_record(const g6x_jrec &r, const JStore &js)
{
    const int a = r.address;
    if (a < 0 || a >= js.cap)
        return;
    js.x0[a] = r.x[0];
    js.x0[js.cap + a] = r.x[1];
    js.x0[2 * js.cap + a] = r.x[2];
    const float hx = __double2float_rn(r.x[0]), hy = __double2float_rn(r.x[1]),
                hz = __double2float_rn(r.x[2]);
    js_xds(js, a) = make_float4(hx, hy, hz, __double2float_rn(r.x[0] - (double)hx));
    js_xds2(js, a) = make_float2(__double2float_rn(r.x[1] - (double)hy),
                             __double2float_rn(r.x[2] - (double)hz));
    js_t0(js, a) = r.tj;
    js_v0m(js, a) = make_float4((float)r.v[0], (float)r.v[1], (float)r.v[2], (float)r.mass);
    js_a2f(js, a) = make_float4((float)r.a2[0], (float)r.a2[1], (float)r.a2[2], 0.f);
    js_j6f(js, a) = make_float4((float)r.j6[0], (float)r.j6[1], (float)r.j6[2], 0.f);
    js.v64[a] = make_double4_32a(r.v[0], r.v[1], r.v[2], r.mass);
    js.a264[a] = make_double4_32a(r.a2[0], r.a2[1], r.a2[2], 0.0);
    js.j664[a] = make_double4_32a(r.j6[0], r.j6[1], r.j6[2], 0.0);
    js.idx[a] = r.index;
    js_idx(js, a) = r.index;
}

// DS + SP addition of Sect. 2.2: (hi, lo) + d with the FP32 operations of a
// TwoSum of hi and d, the low part added in, and a final renormalisation
// (Fast2Sum) -- ten FP32 operations.
__device__ __forceinline__ void ds_add_f(float hi, float lo, float d, float &rh, float &rl)
{
    float s, e;
    two_sum(hi, d, s, e);
    e = __fadd_rn(e, lo);
    rh = __fadd_rn(s, e);
    rl = __fsub_rn(e, __fsub_rn(rh, s));
}

// Eq. 1 and Eq. 2 for one j-slot k < nj, written as the tiled DS layout:
// the paper's form (Sect. 2.2) -- Taylor increment dt (v + dt (a/2 + dt j/6))
// in FP32, added to the double-single x0 by the DS + SP addition, velocity in
// FP32; only dt = t - t0 is formed in FP64 (block times are exact there).
// The DS position part of Eq. 1 (hi, lo per component).
__device__ __forceinline__ void predict_ds_pos(float h, float4 xa, float2 xb, float4 v,
                                               float4 a, float4 j, float *hi, float *lo)
{
    ds_add_f(xa.x, xa.w, h * fmaf(h, fmaf(h, j.x, a.x), v.x), hi[0], lo[0]);
    ds_add_f(xa.y, xb.x, h * fmaf(h, fmaf(h, j.y, a.y), v.y), hi[1], lo[1]);
    ds_add_f(xa.z, xb.y, h * fmaf(h, fmaf(h, j.z, a.z), v.z), hi[2], lo[2]);
}

__device__ __forceinline__ void predict_ds_vals(float h, float4 xa, float2 xb, float4 v,
                                                float4 a, float4 j, int id, float *o)
{
    float hi[3], lo[3];
    predict_ds_pos(h, xa, xb, v, a, j, hi, lo);
    const float h3 = 3.0f * h;
    o[W_XH * JT] = hi[0];
    o[W_YH * JT] = hi[1];
    o[W_ZH * JT] = hi[2];
    o[W_M * JT] = v.w;
    o[W_XL * JT] = lo[0];
    o[W_YL * JT] = lo[1];
    o[W_ZL * JT] = lo[2];
    o[W_VX * JT] = fmaf(h, fmaf(h3, j.x, 2.0f * a.x), v.x);
    o[W_VY * JT] = fmaf(h, fmaf(h3, j.y, 2.0f * a.y), v.y);
    o[W_VZ * JT] = fmaf(h, fmaf(h3, j.z, 2.0f * a.z), v.z);
    o[W_ID * JT] = __int_as_float(id);
}

__device__ __forceinline__ void far_slot_ds(float *o)
{
    o[W_XH * JT] = (float)FAR;
    o[W_YH * JT] = (float)FAR;
    o[W_ZH * JT] = (float)FAR;
    o[W_M * JT] = 0.f;
    o[W_XL * JT] = 0.f;
    o[W_YL * JT] = 0.f;
    o[W_ZL * JT] = 0.f;
    o[W_VX * JT] = 0.f;
    o[W_VY * JT] = 0.f;
    o[W_VZ * JT] = 0.f;
    o[W_ID * JT] = __int_as_float(-1);
}

struct ForceArgs {
    const float *pt;                  // DS predicted j, tiled layout
    const int2 *trange;               // DS per-tile index range
    const double4_32a *p64, *v64;         // FP64 predicted j
    const g6x_irec *irec;
    void *part;                       // PartialDS (DS kernels) or Partial64 (FP64)
    int *nbl;                         // list entries  [slot][nbseg]
    int *nbr;                         // split-j shapes: runs of the j-groups [slot][TJ][nbseg]
    int *nbc;                         // list counts   [slot]
    int maxnb;                        // list length kept per i-particle (Sect. 4)
    int nbseg;                        // entries a list partial has room for (<= maxnb)
    int *nbmax;                       // largest min(count, maxnb) of any list partial
    int *nbl_out, *nblen_out;         // fused reduction: the lists [i][maxnb], their lengths
    int *err;
    long long W;
    int J;
    int ni;
    double eps2;
    // fused reduction: the last CTA to finish an i-tile reduces it into out
    g6x_out *out;
    const int *jidx;
    unsigned *tcnt;                   // per i-tile: CTAs done (0 between launches)
    int fused;
    BatchTables bt;                   // batch geometry (batch kernels only)
    unsigned long long wait_ns;       // limit of each wait for a staged tile
    // prediction inside the force kernel: the j-store, the block time and
    // the number of particles in j-memory; with one i-tile (each j-tile
    // handled by one CTA) also the staged j-records, sorted by tile, that
    // each CTA stores for its own tiles before it reads them
    JStore js;
    double t_pred;
    int nj;
    const g6x_jrec *rec;
    const int *toff;
    // warp-specialised small-block kernel: CTAs per first-level group of its
    // two-level partial reduction (tcnt then holds one counter per group and
    // one for the top level)
    int gs;
};

// Sum of partial records of one i-particle: compensated FP32 for the DS path
// (converted to FP64 once, at the end), plain FP64 for the FP64 path; the
// nearest neighbour is the smallest |r|^2, ties to the lower j-slot.
template <class PT>
struct PartialSum;

template <>
struct PartialSum<PartialDS> {
    float h[7], l[7];
    float br;
    int bj;
    __device__ void init()
    {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            h[q] = 0.f;
            l[q] = 0.f;
        }
        br = __int_as_float(0x7f800000);
        bj = -1;
    }
    __device__ void nn(float r, int j)
    {
        if (j >= 0 && (bj < 0 || r < br || (r == br && j < bj))) {
            br = r;
            bj = j;
        }
    }
    __device__ void add(const PartialDS &P)
    {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ds_acc(h[d], l[d], P.acc[d].x, P.acc[d].y);
            ds_acc(h[3 + d], l[3 + d], P.jerk[d].x, P.jerk[d].y);
        }
        ds_acc(h[6], l[6], P.pot.x, P.pot.y);
        nn(P.nnr2, P.nnj);
    }
    __device__ void shfl_combine(int off)
    {
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const float oh = __shfl_xor_sync(0xffffffffu, h[q], off);
            const float ol = __shfl_xor_sync(0xffffffffu, l[q], off);
            ds_acc(h[q], l[q], oh, ol);
        }
        const float r = __shfl_xor_sync(0xffffffffu, br, off);
        const int j = __shfl_xor_sync(0xffffffffu, bj, off);
        nn(r, j);
    }
    __device__ double value(int q) const { return (double)h[q] + (double)l[q]; }
    __device__ float nnr2() const { return br; }
};

template <>
struct PartialSum<Partial64> {
    double s[7];
    double br;
    int bj;
    __device__ void init()
    {
#pragma unroll
        for (int q = 0; q < 7; ++q)
            s[q] = 0.0;
        br = __longlong_as_double(0x7ff0000000000000ll);
        bj = -1;
    }
    __device__ void nn(double r, int j)
    {
        if (j >= 0 && (bj < 0 || r < br || (r == br && j < bj))) {
            br = r;
            bj = j;
        }
    }
    __device__ void add(const Partial64 &P)
    {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s[d] += P.acc[d];
            s[3 + d] += P.jerk[d];
        }
        s[6] += P.pot;
        nn(P.nnr2, P.nnj);
    }
    __device__ void shfl_combine(int off)
    {
#pragma unroll
        for (int q = 0; q < 7; ++q)
            s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
        const double r = __shfl_xor_sync(0xffffffffu, br, off);
        const int j = __shfl_xor_sync(0xffffffffu, bj, off);
        nn(r, j);
    }
    __device__ double value(int q) const { return s[q]; }
    __device__ float nnr2() const { return (float)br; }
};

template <class PS>
__device__ __forceinline__ g6x_out result_of(const PS &acc, const int *jidx)
{
    g6x_out o;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        o.acc[d] = acc.value(d);
        o.jerk[d] = acc.value(3 + d);
    }
    o.pot = -acc.value(6);
    // a winner that far away is an empty slot (parked at FAR), not a particle:
    // no other j-particle took part
    const bool has_nn = acc.bj >= 0 && acc.nnr2() < 1e30f;
    o.nnb = has_nn ? jidx[acc.bj] : -1;
    o.nnr2 = has_nn ? acc.nnr2() : __int_as_float(0x7f800000);
    return o;
}

// Launch fn, with programmatic stream serialization when pdl is set (the
// kernel then starts behind its predecessor and waits in grid_dep_wait).
template <class... Args>
cudaError_t launch_maybe_pdl(void (*fn)(Args...), int grid, int threads, int smem,
                             cudaStream_t s, bool pdl, Args... args)
{
    if (!pdl) {
        fn<<<grid, threads, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3((unsigned)threads);
    lc.dynamicSmemBytes = (size_t)smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, fn, args...);
}

}  // namespace g6
