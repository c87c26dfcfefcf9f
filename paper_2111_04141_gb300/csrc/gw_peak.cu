// FP32 FMA throughput probe: the achievable packed-FMA (FFMA2) rate of the
// device, a measured cross-check of the nominal FP32 roofline
// (SMs x 128 FMA/clk x 2 FLOP x clock) that the gridder is reported against.
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kChains = 8;   // independent accumulator pairs per thread

__global__ void __launch_bounds__(256) k_ffma_peak(int iters, float seed, float2* out) {
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = make_float2(seed * (threadIdx.x + c), seed * (blockIdx.x - c));
    const float2 m = make_float2(0.999999f, 1.000001f);
    const float2 d = make_float2(1e-7f, -1e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], m, d);
    }
    float2 s = acc[0];
#pragma unroll
    for (int c = 1; c < kChains; ++c) {
        s.x += acc[c].x;
        s.y += acc[c].y;
    }
    if (s.x == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the work
}

}  // namespace

cudaError_t measure_ffma_peak(int num_sms, int iters, double* tflops, cudaStream_t s) {
    float2* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    const int blocks = num_sms * 8, threads = 256;
    cudaError_t e = cudaMalloc(&out, sizeof(float2) * blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        k_ffma_peak<<<blocks, threads, 0, s>>>(iters / 10 + 1, 1e-3f, out);   // warm-up
        cudaEventRecord(a, s);
        k_ffma_peak<<<blocks, threads, 0, s>>>(iters, 1e-3f, out);
        cudaEventRecord(b, s);
        note_launch(2);
        e = cudaEventSynchronize(b);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess)
        *tflops = (double)blocks * threads * iters * kChains * 4.0 / (ms * 1e-3) / 1e12;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    return e;
}

}  // namespace gw
