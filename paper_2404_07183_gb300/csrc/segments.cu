// segments.cu -- single-PCF functionals by segment iteration (Sec. 3.2, Alg. 3).
//
// out[i] = r( int_a^b h(f_i(t)) dt ) with h(v) = v (the integral of f) or
// h(v) = |v|^p (r = x^(1/p) when requested: the L_p norm).  A PCF's segments
// [t_k, t_{k+1}) (the last one reaching inf) are clipped to [a, b]; one warp
// takes one PCF, lane l the segments l, l + 32, ...; the float64 partial sums
// are combined in a fixed lane order.  A last segment reaching b = inf adds 0
// when h = 0 and h * inf otherwise.
#include <cmath>

#include "internal.cuh"

namespace pcfgb {

__device__ __forceinline__ double seg_pow(double v, double p)
{
    const double a = fabs(v);
    if (p == 1.0) return a;
    if (p == 2.0) return v * v;
    if (p == 3.0) return a * a * a;
    return pow(a, p);
}

template <typename Tin>
__global__ void segment_kernel(const int64_t* __restrict__ offsets, const Tin* __restrict__ times,
                               const Tin* __restrict__ values, int64_t n, int functional, double p,
                               int apply_root, double lo, double hi, void* out, int out_f64,
                               const Header* hdr)
{
    if (hdr->err != kNoError) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < n; i += nwarps) {
        const int64_t o0 = offsets[i], o1 = offsets[i + 1];
        double acc = 0.0;
        bool diverges = false;
        double tail_sign = 0.0;
        for (int64_t k = o0 + lane; k < o1; k += 32) {
            const double v = (double)values[k];
            const double h = functional == PCF_FN_INTEGRAL ? v : seg_pow(v, p);
            const double l = fmax((double)times[k], lo);
            const double r = fmin((k + 1 < o1) ? (double)times[k + 1] : (double)INFINITY, hi);
            if (!(r > l)) continue;
            if (isinf(r)) {
                if (h != 0.0) { diverges = true; tail_sign = h > 0.0 ? 1.0 : -1.0; }
                continue;
            }
            acc = fma(h, r - l, acc);
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
        const unsigned div = __ballot_sync(0xffffffffu, diverges);
        double sign = 0.0;
        if (div) sign = __shfl_sync(0xffffffffu, tail_sign, __ffs(div) - 1);
        if (lane == 0) {
            double I = div ? sign * (double)INFINITY : acc;
            if (apply_root && functional == PCF_FN_LP && p != 1.0)
                I = (p == 2.0) ? sqrt(I) : pow(I, 1.0 / p);
            if (out_f64) reinterpret_cast<double*>(out)[i] = I;
            else reinterpret_cast<float*>(out)[i] = (float)I;
        }
    }
}

cudaError_t launch_segments(const pcf_csr* x, int functional, double p, int apply_root,
                            double lo, double hi, void* out, int out_f64, const Header* hdr,
                            cudaStream_t s)
{
    if (x->n == 0) return cudaSuccess;
    int64_t blocks = (x->n * 32 + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (x->dtype == PCF_F64)
        segment_kernel<double><<<(int)blocks, 256, 0, s>>>(x->offsets, (const double*)x->times,
            (const double*)x->values, x->n, functional, p, apply_root, lo, hi, out, out_f64, hdr);
    else
        segment_kernel<float><<<(int)blocks, 256, 0, s>>>(x->offsets, (const float*)x->times,
            (const float*)x->values, x->n, functional, p, apply_root, lo, hi, out, out_f64, hdr);
    return cudaGetLastError();
}

}  // namespace pcfgb
