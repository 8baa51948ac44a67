// Arithmetic peak of the current device, measured: the denominator of the
// FP32 and FP64 roofline fractions the benchmark reports for the near and far
// fields.  Every thread runs kChains independent FMA chains (a <- a * b + c)
// for a fixed number of steps; the grid holds kBlocksPerSm blocks of 256
// threads per SM, so every FMA pipe of every SM has independent work at every
// cycle.  FP32 is measured both with scalar FMAs and with packed FP32x2 FMAs
// (two lanes of work per instruction, the form the near and far kernels use)
// and the faster of the two is reported.
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kBlocksPerSm = 8;

// a sink no run can hit (the chains stay finite and far from it), so the
// compiler must keep every FMA
__device__ float g_probe_sink32;
__device__ double g_probe_sink64;

__global__ void __launch_bounds__(kProbeThreads) k_probe_f32(int steps, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < steps; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.2345e30f) g_probe_sink32 = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_f32x2(int steps, float b, float c)
{
    float2 a[kChains / 2];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
    for (int k = 0; k < kChains / 2; k++) a[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
    for (int i = 0; i < steps; i++) {
#pragma unroll
        for (int k = 0; k < kChains / 2; k++) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; k++) s += a[k].x + a[k].y;
    if (s == -1.2345e30f) g_probe_sink32 = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_f64(int steps, double b, double c)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < steps; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.2345e300) g_probe_sink64 = s;
}

}  // namespace

// Best of `reps` timed launches (after one warm-up) of one probe kernel;
// flops per launch = 2 * kChains * steps * threads.
cudaError_t run_probe(int kind, cudaStream_t s, double* tflops, double* ms_best)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)(sms * kBlocksPerSm);
    // about 1 ms per launch at the nominal rates
    const int steps = kind == 2 ? 256 : 16384;
    const double flops = 2.0 * kChains * (double)steps * grid * kProbeThreads;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    const int reps = 5;
    for (int r = 0; r <= reps && e == cudaSuccess; r++) {
        e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) break;
        if (kind == 0)
            k_probe_f32<<<grid, kProbeThreads, 0, s>>>(steps, 0.999999f, 1e-6f);
        else if (kind == 1)
            k_probe_f32x2<<<grid, kProbeThreads, 0, s>>>(steps, 0.999999f, 1e-6f);
        else
            k_probe_f64<<<grid, kProbeThreads, 0, s>>>(steps, 0.999999999, 1e-9);
        note_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && r > 0 && (best == 0.f || t < best)) best = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    *ms_best = best;
    *tflops = flops / (best * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace tc
