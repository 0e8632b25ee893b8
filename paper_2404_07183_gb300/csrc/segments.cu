// segments.cu -- single-PCF functionals by segment iteration (Sec. 3.2, Alg. 3).
//
// out[i] = r( int_a^b h(f_i(t)) dt ) with h(v) = v (the integral of f) or
// h(v) = |v|^p (r = x^(1/p) when requested: the L_p norm).  A PCF's segments
// [t_k, t_{k+1}) (the last one reaching inf) are clipped to [a, b]; one warp
// takes one PCF, lane l the segments l, l + 32, ...; the lane partial sums are
// combined in float64 in a fixed lane order.  Arithmetic per segment: float64
// (PCF_PREC_F64), or float32 on float32 data with Kahan's compensated
// summation per segment (PCF_PREC_F32_COMP; float64 data are rounded to
// float32 first).  A last segment reaching b = inf adds 0 when h = 0 and
// h * inf otherwise.
#include <cmath>

#include "internal.cuh"

namespace pcfgb {

template <typename T>
__device__ __forceinline__ T seg_pow(T v, T p)
{
    const T a = fabs(v);
    if (p == T(1)) return a;
    if (p == T(2)) return v * v;
    if (p == T(3)) return a * a * a;
    return pow(a, p);
}

// Per-lane accumulator: float64 fma, or float32 Kahan (sum - compensation).
template <typename T> struct SegAcc;
template <> struct SegAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double h, double len) { s = fma(h, len, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct SegAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float h, float len)
    {
        const float y = __fmaf_rn(h, len, -c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename Tin, typename T>
__global__ void segment_kernel(const int64_t* __restrict__ offsets, const Tin* __restrict__ times,
                               const Tin* __restrict__ values, int64_t n, int functional, double p_,
                               int apply_root, double lo_, double hi_, void* out, int out_f64,
                               const Header* hdr)
{
    const T p = (T)p_, lo = (T)lo_, hi = (T)hi_;
    if (hdr->err != kNoError) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < n; i += nwarps) {
        const int64_t o0 = offsets[i], o1 = offsets[i + 1];
        SegAcc<T> sa;
        bool diverges = false;
        double tail_sign = 0.0;
        for (int64_t k = o0 + lane; k < o1; k += 32) {
            const T v = (T)values[k];
            const T h = functional == PCF_FN_INTEGRAL ? v : seg_pow<T>(v, p);
            const T t0 = (T)times[k];
            const T t1 = (k + 1 < o1) ? (T)times[k + 1] : T(INFINITY);
            const T l = t0 > lo ? t0 : lo;
            const T r = t1 < hi ? t1 : hi;
            if (!(r > l)) continue;
            if (isinf(r)) {
                if (h != T(0)) { diverges = true; tail_sign = h > T(0) ? 1.0 : -1.0; }
                continue;
            }
            sa.add(h, r - l);
        }
        double acc = sa.value();
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
        const unsigned div = __ballot_sync(0xffffffffu, diverges);
        double sign = 0.0;
        if (div) sign = __shfl_sync(0xffffffffu, tail_sign, __ffs(div) - 1);
        if (lane == 0) {
            double I = div ? sign * (double)INFINITY : acc;
            if (apply_root && functional == PCF_FN_LP && p_ != 1.0)
                I = (p_ == 2.0) ? sqrt(I) : pow(I, 1.0 / p_);
            if (out_f64) reinterpret_cast<double*>(out)[i] = I;
            else reinterpret_cast<float*>(out)[i] = (float)I;
        }
    }
}

cudaError_t launch_segments(const pcf_csr* x, int functional, double p, int apply_root,
                            double lo, double hi, int precision, void* out, int out_f64,
                            const Header* hdr, cudaStream_t s)
{
    if (x->n == 0) return cudaSuccess;
    int64_t blocks = (x->n * 32 + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    const bool f32 = precision != PCF_PREC_F64;
#define PCF_SEG_LAUNCH(TIN, TW)                                                               \
    segment_kernel<TIN, TW><<<(int)blocks, 256, 0, s>>>(x->offsets, (const TIN*)x->times,      \
        (const TIN*)x->values, x->n, functional, p, apply_root, lo, hi, out, out_f64, hdr)
    if (x->dtype == PCF_F64) {
        if (f32) PCF_SEG_LAUNCH(double, float); else PCF_SEG_LAUNCH(double, double);
    } else {
        if (f32) PCF_SEG_LAUNCH(float, float); else PCF_SEG_LAUNCH(float, double);
    }
#undef PCF_SEG_LAUNCH
    return cudaGetLastError();
}

}  // namespace pcfgb
