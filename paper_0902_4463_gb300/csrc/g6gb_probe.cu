// g6gb_probe.cu -- FP32 throughput probe.
//
// The force kernel is bound by the FP32 pipe, and its roofline denominator is
// derived from the unit counts and the clock (SMs x 128 FP32 lanes x 2 flop x
// f_SM).  This probe measures what that pipe delivers: every thread runs
// independent chains of packed FP32x2 fused multiply-adds (the instruction
// form of the force kernel's pair loop), with enough resident warps on every
// SM to hide the dependent latency, and the kernel is timed with CUDA events.
// It is a measurement, not part of the force path; it allocates a small
// output buffer and leaves no state behind.
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

}  // namespace

extern "C" int g6x_fp32_probe(int iters, double *tflops, double *ms)
{
    if (iters < 1 || iters > (1 << 24) || !tflops)
        return G6_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess
        || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess
        || sms < 1) {
        cudaGetLastError();
        return G6_ENODEV;
    }
    const int grid = sms * PROBE_CTAS_PER_SM;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    float elapsed = 0.0f;
    const float2 a = make_float2(0.999f, 0.998f), b = make_float2(1e-3f, 2e-3f);
    if (cudaMalloc(&out, sizeof(float) * (size_t)grid * PROBE_THREADS) != cudaSuccess
        || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess
        || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = G6_ENOMEM;
    } else {
        // one short warm-up launch, then the timed one
        k_fp32_probe<<<grid, PROBE_THREADS, 0, st>>>(out, iters / 16 + 1, a, b, -1.0f);
        cudaEventRecord(e0, st);
        k_fp32_probe<<<grid, PROBE_THREADS, 0, st>>>(out, iters, a, b, -1.0f);
        cudaEventRecord(e1, st);
        if (cudaStreamSynchronize(st) != cudaSuccess
            || cudaEventElapsedTime(&elapsed, e0, e1) != cudaSuccess || !(elapsed > 0.0f))
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
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    // per thread and loop trip: UNROLL x CHAINS packed FMAs = 2 lanes x 2 flop each
    const double flop = 4.0 * PROBE_UNROLL * PROBE_CHAINS * (double)iters * grid * PROBE_THREADS;
    *tflops = flop / (elapsed * 1e-3) / 1e12;
    if (ms)
        *ms = elapsed;
    return 0;
}
