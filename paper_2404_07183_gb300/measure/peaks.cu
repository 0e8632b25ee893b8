// peaks.cu -- arithmetic-pipe microbenchmarks that set the roofline
// denominators of the merge walk (measurement code; not part of the library).
//
// Each kernel runs one 1024-thread block per SM; every thread keeps eight
// independent fused-multiply-add chains for `iters` rounds.  Thread 0 of each
// block reads the SM cycle counter around the loop, so the result is lane
// operations per SM per clock, independent of the clock the GPU ran at.
#include <cstdint>
#include <cuda_runtime.h>

template <typename T>
__global__ void __launch_bounds__(1024, 1) fma_chains(T* out, long long* cycles, int iters, T b, T c)
{
    T a0 = (T)threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    T a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    __syncthreads();
    long long t0 = clock64();
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    __syncthreads();
    long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

extern "C" int pcf_peak_fma(int use_f64, int blocks, int iters, double* lane_ops_per_clk,
                            double* lane_ops_per_s)
{
    void* out = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * 1024 * 8) != cudaSuccess) return 1;
    if (cudaMalloc((void**)&cyc, (size_t)blocks * sizeof(long long)) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        if (use_f64) fma_chains<double><<<blocks, 1024>>>((double*)out, cyc, iters, 0.999999, 1e-7);
        else fma_chains<float><<<blocks, 1024>>>((float*)out, cyc, iters, 0.9999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    long long* h = new long long[blocks];
    cudaMemcpy(h, cyc, (size_t)blocks * sizeof(long long), cudaMemcpyDeviceToHost);
    // median block cycle count
    for (int i = 1; i < blocks; ++i)
        for (int j = i; j > 0 && h[j - 1] > h[j]; --j) { long long x = h[j]; h[j] = h[j - 1]; h[j - 1] = x; }
    const double ops_per_block = 1024.0 * 8.0 * (double)iters;
    *lane_ops_per_clk = ops_per_block / (double)h[blocks / 2];
    *lane_ops_per_s = ops_per_block * blocks / (ms * 1e-3);
    delete[] h;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
