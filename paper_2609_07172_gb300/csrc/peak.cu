// FMA throughput probe: the ALU roofline denominators for kernels bound by
// FP64 arithmetic.  Every thread runs NCHAIN independent FMA chains held in
// registers (no memory traffic inside the loop); the grid fills every SM.
#include "internal.h"

namespace pp {
namespace {

constexpr int NCHAIN = 8;
constexpr int PEAK_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma(T *out, int iters, T a, T b) {
    T x[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < NCHAIN; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += x[c];
    if (s == (T)12345.678) out[0] = s;   // keeps the chains live; practically never taken
}

template <class T>
cudaError_t time_one(cudaStream_t st, int iters, double *gflops) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    T *out = nullptr;
    cudaError_t err = cudaMallocAsync((void **)&out, sizeof(T), st);
    if (err != cudaSuccess) return err;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const T ca = (T)0.999999, cb = (T)1e-7;
    k_fma<T><<<blocks, PEAK_THREADS, 0, st>>>(out, iters / 8, ca, cb);   // warm-up
    cudaEventRecord(a, st);
    k_fma<T><<<blocks, PEAK_THREADS, 0, st>>>(out, iters, ca, cb);
    cudaEventRecord(b, st);
    err = cudaEventSynchronize(b);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(out, st);
    if (err != cudaSuccess) return err;
    const double flops = 2.0 * NCHAIN * 16.0 * (double)iters * (double)blocks * PEAK_THREADS;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return cudaGetLastError();
}

}  // namespace

cudaError_t measure_fma(cudaStream_t st, double *fp64_gflops, double *fp32_gflops) {
    cudaError_t e = time_one<double>(st, 256, fp64_gflops);
    if (e != cudaSuccess) return e;
    return time_one<float>(st, 8192, fp32_gflops);
}

}  // namespace pp
