// FP64 / FP32 FMA throughput probe: the denominator of the arithmetic roofline of the J-engine.
// Eight independent FMA chains per thread, a grid of 4 blocks x 256 threads per SM, timed with CUDA
// events after a warm-up launch.  The SM clock is estimated from clock64() over the timed launch.
#include <cuda_runtime.h>

#include "internal.hpp"

namespace fef {

template <typename T>
__global__ void k_fma_chain(T* out, long long* cycles, int iters, T a, T b)
{
    long long c0 = clock64();
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (blockIdx.x == 0 && threadIdx.x == 0) *cycles = clock64() - c0;
}

template <typename T>
static cudaError_t run_probe(int sms, int iters, double* flops, double* mhz)
{
    const int blocks = sms * 4, threads = 256;
    T* out = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&out, sizeof(T) * blocks * threads);
    if (err == cudaSuccess) err = cudaMalloc(&cyc, sizeof(long long));
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) {
        k_fma_chain<T><<<blocks, threads>>>(out, cyc, iters / 8, (T)0.999999, (T)1e-7);
        note_launches(1);
        cudaEventRecord(e0);
        k_fma_chain<T><<<blocks, threads>>>(out, cyc, iters, (T)0.999999, (T)1e-7);
        note_launches(1);
        cudaEventRecord(e1);
        err = cudaEventSynchronize(e1);
    }
    if (err == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        long long c = 0;
        cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
        double fma_total = (double)blocks * threads * iters * 8.0;
        if (flops) *flops = 2.0 * fma_total / (ms * 1e-3);
        if (mhz) *mhz = (double)c / (ms * 1e-3) / 1e6;
        err = cudaGetLastError();
    }
    if (out) cudaFree(out);
    if (cyc) cudaFree(cyc);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return err;
}

cudaError_t measure_fma_peak(double* fp64, double* fp32, double* mhz)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    double m64 = 0, m32 = 0;
    e = run_probe<double>(sms, 1 << 14, fp64, &m64);
    if (e == cudaSuccess) e = run_probe<float>(sms, 1 << 19, fp32, &m32);
    if (mhz) *mhz = m64;
    return e;
}

}  // namespace fef
