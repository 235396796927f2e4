// g6gb_probe.cu -- FP32 and FP64 throughput probes.
//
// The force kernel is bound by the FP32 pipe, and its roofline denominator is
// derived from the unit counts and the clock (SMs x 128 FP32 lanes x 2 flop x
// f_SM).  The FP32 probe measures what that pipe delivers: every thread runs
// independent chains of packed FP32x2 fused multiply-adds (the instruction
// form of the force kernel's pair loop), with enough resident warps on every
// SM to hide the dependent latency, and the kernel is timed with CUDA events.
// The FP64 probe does the same with FP64 fused multiply-adds: it is the
// roofline denominator of the all-FP64 force kernel, the comparison kernel of
// the precision argument (Sect. 2.3).  They are measurements, not part of the
// force path; each allocates a small output buffer and leaves no state behind.
#include "g6gb_internal.h"

#include <cuda_runtime.h>

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent chains per thread
constexpr int PROBE_UNROLL = 16;  // FMAs per chain per loop trip
constexpr int PROBE_CTAS_PER_SM = 8;

// acc <- acc * a + b on every chain; with 0 < a < 1 the values converge to
// b / (1 - a) and stay normal.  The sum is written only if it equals a value
// it never takes, so the work cannot be removed and nothing is stored.
__global__ void __launch_bounds__(PROBE_THREADS) k_fp32_probe(float *out, int iters, float2 a,
                                                              float2 b, float never)
{
    float2 acc[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c)
        acc[c] = make_float2(1e-3f * (float)(threadIdx.x & 31) + (float)c, 0.5f * (float)c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c)
                acc[c] = __ffma2_rn(acc[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c)
        s += acc[c].x + acc[c].y;
    if (s == never)
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same with FP64 fused multiply-adds (scalar: there is no packed FP64).
constexpr int PROBE64_CHAINS = 8;
__global__ void __launch_bounds__(PROBE_THREADS) k_fp64_probe(double *out, int iters, double a,
                                                              double b, double never)
{
    double acc[PROBE64_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE64_CHAINS; ++c)
        acc[c] = 1e-3 * (double)(threadIdx.x & 31) + (double)c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < PROBE64_CHAINS; ++c)
                acc[c] = fma(acc[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PROBE64_CHAINS; ++c)
        s += acc[c];
    if (s == never)
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Time one launch of kern (after a short warm-up launch of it) with CUDA
// events on a stream of its own; fills *elapsed in ms.
template <class T, class K, class A, class B>
int time_probe(K kern, int iters, A a, A b, B never, float *elapsed)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess
        || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess
        || sms < 1) {
        cudaGetLastError();
        return G6_ENODEV;
    }
    const int grid = sms * PROBE_CTAS_PER_SM;
    T *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    *elapsed = 0.0f;
    if (cudaMalloc(&out, sizeof(T) * (size_t)grid * PROBE_THREADS) != cudaSuccess
        || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess
        || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = G6_ENOMEM;
    } else {
        kern<<<grid, PROBE_THREADS, 0, st>>>(out, iters / 16 + 1, a, b, never);
        cudaEventRecord(e0, st);
        kern<<<grid, PROBE_THREADS, 0, st>>>(out, iters, a, b, never);
        cudaEventRecord(e1, st);
        if (cudaStreamSynchronize(st) != cudaSuccess
            || cudaEventElapsedTime(elapsed, e0, e1) != cudaSuccess || !(*elapsed > 0.0f))
            rc = G6_EIO;
    }
    if (e1)
        cudaEventDestroy(e1);
    if (e0)
        cudaEventDestroy(e0);
    if (st)
        cudaStreamDestroy(st);
    if (out)
        cudaFree(out);
    if (rc)
        cudaGetLastError();
    return rc ? rc : grid;
}

}  // namespace

extern "C" int g6x_fp64_probe(int iters, double *tflops, double *ms)
{
    if (iters < 1 || iters > (1 << 24) || !tflops)
        return G6_EINVAL;
    float elapsed = 0.0f;
    const int grid = time_probe<double>(k_fp64_probe, iters, 0.999, 1e-3, -1.0, &elapsed);
    if (grid < 0)
        return grid;
    // per thread and loop trip: UNROLL x CHAINS FMAs of 2 flop each
    const double flop = 2.0 * PROBE_UNROLL * PROBE64_CHAINS * (double)iters * grid * PROBE_THREADS;
    *tflops = flop / (elapsed * 1e-3) / 1e12;
    if (ms)
        *ms = elapsed;
    return 0;
}

extern "C" int g6x_fp32_probe(int iters, double *tflops, double *ms)
{
    if (iters < 1 || iters > (1 << 24) || !tflops)
        return G6_EINVAL;
    float elapsed = 0.0f;
    const int grid = time_probe<float>(k_fp32_probe, iters, make_float2(0.999f, 0.998f),
                                       make_float2(1e-3f, 2e-3f), -1.0f, &elapsed);
    if (grid < 0)
        return grid;
    // per thread and loop trip: UNROLL x CHAINS packed FMAs = 2 lanes x 2 flop each
    const double flop = 4.0 * PROBE_UNROLL * PROBE_CHAINS * (double)iters * grid * PROBE_THREADS;
    *tflops = flop / (elapsed * 1e-3) / 1e12;
    if (ms)
        *ms = elapsed;
    return 0;
}
