// fp32_probe.cu -- measures the FP32 FMA throughput of the GPU (the denominator of the
// projector kernels' roofline, which are bound by FP32 arithmetic and instruction issue,
// not by HBM or tensor cores). Built as its own small library, used only by bench.py.
//
// Each thread runs 8 independent chains of dependent FMAs (x = x * m + c), enough
// independent work per scheduler to hide the FMA latency; the grid fills every SM.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) ffma_chains(float* out, int iters, float m, float c) {
    float a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = (float)(threadIdx.x + q) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int q = 0; q < kChains; ++q) a[q] = fmaf(a[q], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    // never true for the arguments bench.py passes; keeps the chains alive
    if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// FP32 FLOP/s (2 per FMA) of one timed launch after one warm-up launch on the current
// device; blocks_per_sm x SMs blocks of 256 threads, `iters` x 128 FMAs per thread.
// Returns 0 on success, the CUDA error code otherwise. Synchronises the device.
int kct_probe_fp32(int blocks_per_sm, int iters, double* flops, float* ms) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    float* out = nullptr;
    e = cudaMalloc(&out, sizeof(float) * (size_t)sms * blocks_per_sm * kThreads);
    if (e != cudaSuccess) return (int)e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const dim3 grid((unsigned)(sms * blocks_per_sm));
    ffma_chains<<<grid, kThreads>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e0);
    ffma_chains<<<grid, kThreads>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double fmas = (double)grid.x * kThreads * (double)iters * kUnroll * kChains;
    *flops = 2.0 * fmas / (t * 1e-3);
    *ms = t;
    return 0;
}

}  // extern "C"
