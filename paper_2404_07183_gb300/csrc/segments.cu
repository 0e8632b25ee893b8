// segments.cu -- single-PCF functionals by segment iteration (Sec. 3.2, Alg. 3).
//
// out[i] = r( int_a^b h(f_i(t)) dt ) with h(v) = v (the integral of f) or
// h(v) = |v|^p (r = x^(1/p) when requested: the L_p norm).  A PCF's segments
// [t_k, t_{k+1}) (the last one reaching inf) are clipped to [a, b].  A warp
// takes a PCF of at most 1024 breakpoints (lane l: segments l, l + 32, ...),
// a CTA takes a longer one (thread t: segments t, t + 256, ...), so the
// longest PCFs no longer set the kernel time; partial sums are combined in
// float64 in a fixed order.  The input is checked in the same pass, with the
// reasons and indices of pcf_pairwise's check.  Arithmetic per segment: float64
// (PCF_PREC_F64), or float32 on float32 data with Kahan's compensated
// summation per segment (PCF_PREC_F32_COMP; float64 data are rounded to
// float32 first).  A last segment reaching b = inf adds 0 when h = 0 and
// h * inf otherwise.
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace pcfgb {

// Integrand h(v) of the functional, fixed at compile time.
enum SegFn : int { kFnIntegral = 0, kFnAbs = 1, kFnSquare = 2, kFnCube = 3, kFnPow = 4 };

template <int FN, typename T>
__device__ __forceinline__ T seg_h(T v, T p)
{
    if constexpr (FN == kFnIntegral) return v;
    else if constexpr (FN == kFnAbs) return fabs(v);
    else if constexpr (FN == kFnSquare) return v * v;
    else if constexpr (FN == kFnCube) { const T a = fabs(v); return a * a * a; }
    else return pow(fabs(v), p);
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

// Sum of the 32 lanes' accumulators into lane 0's (fixed tree order).
// float64: plain float64 additions.  float32: the lanes' (sum, compensation)
// pairs are merged with Knuth's error-free TwoSum of the sums, the rounding
// error joining the compensation, so every step stays on the FP32 pipe (the
// FP64 pipe of GB300 is narrow) and the compensated error bound holds.
__device__ __forceinline__ void seg_warp_reduce(SegAcc<double>& a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a.s += __shfl_down_sync(0xffffffffu, a.s, o);
}
__device__ __forceinline__ void seg_warp_reduce(SegAcc<float>& a)
{
    float s = a.s, c = a.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o);
        const float c2 = __shfl_down_sync(0xffffffffu, c, o);
        const float t = __fadd_rn(s, s2);                      // TwoSum(s, s2): t + e exactly
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2), e);                    // value = s - c
    }
    a.s = s; a.c = c;
}
// Lane 0's accumulator in every lane.
__device__ __forceinline__ SegAcc<double> seg_lane0(const SegAcc<double>& a)
{
    SegAcc<double> r; r.s = __shfl_sync(0xffffffffu, a.s, 0); return r;
}
__device__ __forceinline__ SegAcc<float> seg_lane0(const SegAcc<float>& a)
{
    SegAcc<float> r;
    r.s = __shfl_sync(0xffffffffu, a.s, 0);
    r.c = __shfl_sync(0xffffffffu, a.c, 0);
    return r;
}

constexpr int64_t kSegLong = 1024;   // longer PCFs get a whole CTA
constexpr int kSegUnroll = 4;        // elements in flight per thread

// One segment [t_k, t_{k+1}) of PCF i: validate element k as the input check
// of pcf_pairwise does (same reasons, same indices), then add its term.
template <typename Tin, typename T>
struct SegCtx {
    const Tin* times; const Tin* values;
    int functional; T p, lo, hi;
    Header* hdr;
    bool range32;                  // float64 data walked in float32
    bool clip;                     // [a, b] is not [0, inf)
};

// Breakpoint data of one segment, loaded before any check runs so that the
// loads of a whole batch are in flight together.
template <typename Tin>
struct SegLoad { Tin tk, vk, tp, tn; };

template <typename Tin, typename T>
__device__ __forceinline__ SegLoad<Tin> seg_load(const SegCtx<Tin, T>& c, int64_t k, int64_t o0,
                                                 int64_t o1)
{
    SegLoad<Tin> d;
    d.tk = __ldg(c.times + k);
    d.vk = __ldg(c.values + k);
    d.tp = k > o0 ? __ldg(c.times + k - 1) : Tin(0);
    d.tn = k + 1 < o1 ? __ldg(c.times + k + 1) : Tin(INFINITY);
    return d;
}

template <int FN, typename Tin, typename T>
__device__ __forceinline__ void seg_element(const SegCtx<Tin, T>& c, const SegLoad<Tin>& d,
                                            int64_t k, int64_t o0, SegAcc<T>& sa,
                                            bool& diverges, double& tail_sign)
{
    if (!isfinite(d.tk)) { record_error(c.hdr, kErrTimeNaN, k); return; }
    if (!isfinite(d.vk)) { record_error(c.hdr, kErrValueNaN, k); return; }
    if (k == o0) {
        if (d.tk != Tin(0)) record_error(c.hdr, kErrT0, k);
    } else if (!(d.tk > d.tp)) {
        record_error(c.hdr, kErrOrder, k);
    }
    if (c.range32 &&
        (fabs((double)d.tk) > (double)FLT_MAX || fabs((double)d.vk) > (double)FLT_MAX))
        record_error(c.hdr, kErrRange32, k);
    const T v = (T)d.vk;
    const T h = seg_h<FN, T>(v, c.p);
    T l = (T)d.tk, r = (T)d.tn;
    if (c.clip) {
        l = l > c.lo ? l : c.lo;
        r = r < c.hi ? r : c.hi;
        if (!(r > l)) return;
    }
    if (isinf(r)) {
        if (h != T(0)) { diverges = true; tail_sign = h > T(0) ? 1.0 : -1.0; }
        return;
    }
    sa.add(h, r - l);
}

// Segments k0, k0 + step, ... (kSegUnroll of them) of one PCF: loads first.
template <int FN, typename Tin, typename T>
__device__ __forceinline__ void seg_batch(const SegCtx<Tin, T>& c, int64_t k0, int64_t step,
                                          int64_t o0, int64_t o1, SegAcc<T>& sa, bool& diverges,
                                          double& tail_sign)
{
    SegLoad<Tin> d[kSegUnroll];
#pragma unroll
    for (int u = 0; u < kSegUnroll; ++u) {
        const int64_t k = k0 + step * u;
        if (k < o1) d[u] = seg_load(c, k, o0, o1);
    }
#pragma unroll
    for (int u = 0; u < kSegUnroll; ++u) {
        const int64_t k = k0 + step * u;
        if (k < o1) seg_element<FN>(c, d[u], k, o0, sa, diverges, tail_sign);
    }
}

// Offsets of PCF i as pcf_pairwise's input check reads them; false if bad.
__device__ __forceinline__ bool seg_offsets(const int64_t* offsets, int64_t i, int64_t n,
                                            int64_t nnz, Header* hdr, int64_t& o0, int64_t& o1)
{
    o0 = offsets[i]; o1 = offsets[i + 1];
    bool bad = !(o0 >= 0 && o1 > o0 && o1 <= nnz && (o1 - o0) < (1ll << 31));
    if (i == 0 && o0 != 0) bad = true;
    if (i == n - 1 && o1 != nnz) bad = true;
    if (bad) record_error(hdr, kErrOffsets, i);
    return !bad;
}

__device__ __forceinline__ double seg_finish(double acc, bool div, double sign, int functional,
                                             int apply_root, double p)
{
    double I = div ? sign * (double)INFINITY : acc;
    if (apply_root && functional == PCF_FN_LP && p != 1.0)
        I = (p == 2.0) ? sqrt(I) : pow(I, 1.0 / p);
    return I;
}

__device__ __forceinline__ void seg_store(void* out, int out_f64, int64_t i, double I)
{
    if (out_f64) reinterpret_cast<double*>(out)[i] = I;
    else reinterpret_cast<float*>(out)[i] = (float)I;
}

// One warp per PCF of at most kSegLong breakpoints, lane l taking the
// segments l, l + 32, ... (kSegUnroll loads in flight); longer PCFs go on a
// list for segment_long_kernel.  The input check runs on the same loads.
template <typename Tin, typename T, int FN>
__global__ void segment_kernel(const int64_t* __restrict__ offsets, SegCtx<Tin, T> c, int64_t n,
                               int64_t nnz, int apply_root, double p_, void* out, int out_f64,
                               int32_t* long_list)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // float64 form: finished PCFs wait in the lanes (lane j holds the j-th)
    // and are rooted and stored 32 at a time, one warp-wide pass of the
    // float64 finish instead of one per PCF (measured: 0.72 -> 0.66 ms on the
    // log-normal set; the float32 form is faster finishing each PCF in lane 0)
    constexpr bool kBatch = sizeof(T) == 8;
    SegAcc<T> held;
    int64_t held_i = -1;
    double held_sign = 0.0;
    int slot = 0;
    auto flush = [&]() {
        if (held_i >= 0)
            seg_store(out, out_f64, held_i, seg_finish(held.value(), held_sign != 0.0, held_sign,
                                                       c.functional, apply_root, p_));
        held_i = -1;
        slot = 0;
    };
    for (int64_t i = warp0; i < n; i += nwarps) {
        int64_t o0, o1;
        if (!seg_offsets(offsets, i, n, nnz, c.hdr, o0, o1)) continue;
        if (o1 - o0 > kSegLong) {
            if (lane == 0) long_list[atomicAdd(&c.hdr->tiles, 1ull)] = (int32_t)i;
            continue;
        }
        SegAcc<T> sa;
        bool diverges = false;
        double tail_sign = 0.0;
        for (int64_t k0 = o0 + lane; k0 < o1; k0 += 32 * kSegUnroll)
            seg_batch<FN>(c, k0, 32, o0, o1, sa, diverges, tail_sign);
        seg_warp_reduce(sa);
        const SegAcc<T> tot = seg_lane0(sa);
        const unsigned div = __ballot_sync(0xffffffffu, diverges);
        double sign = 0.0;
        if (div) sign = __shfl_sync(0xffffffffu, tail_sign, __ffs(div) - 1);
        if constexpr (kBatch) {
            if (lane == slot) { held = tot; held_i = i; held_sign = sign; }
            if (++slot == 32) flush();
        } else if (lane == 0) {
            seg_store(out, out_f64, i, seg_finish(tot.value(), div != 0, sign, c.functional,
                                                  apply_root, p_));
        }
    }
    if constexpr (kBatch) flush();
}

// One CTA per listed long PCF; thread partial sums combined in a fixed
// order (warp shuffles, then the 8 warp sums in order).
template <typename Tin, typename T, int FN>
__global__ void __launch_bounds__(256) segment_long_kernel(const int64_t* __restrict__ offsets,
                                                           SegCtx<Tin, T> c, int apply_root,
                                                           double p_, void* out, int out_f64,
                                                           const int32_t* long_list)
{
    __shared__ double sAcc[8];
    __shared__ int sDiv[8];
    __shared__ double sSign[8];
    // no early exit on a recorded error: these PCFs' elements still have to
    // be checked so that the smallest offending index is the one reported
    const long long count = (long long)c.hdr->tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long w = blockIdx.x; w < count; w += gridDim.x) {
        const int64_t i = long_list[w];
        const int64_t o0 = offsets[i], o1 = offsets[i + 1];
        SegAcc<T> sa;
        bool diverges = false;
        double tail_sign = 0.0;
        for (int64_t k0 = o0 + threadIdx.x; k0 < o1; k0 += 256 * kSegUnroll)
            seg_batch<FN>(c, k0, 256, o0, o1, sa, diverges, tail_sign);
        seg_warp_reduce(sa);
        const double acc = sa.value();
        const unsigned div = __ballot_sync(0xffffffffu, diverges);
        if (lane == 0) {
            sAcc[warp] = acc;
            sDiv[warp] = div != 0;
            sSign[warp] = 0.0;
        }
        if (div) {                                  // (div is the same in every lane)
            const double sg = __shfl_sync(0xffffffffu, tail_sign, __ffs(div) - 1);
            if (lane == 0) sSign[warp] = sg;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0, sign = 0.0;
            bool any = false;
            for (int q = 0; q < 8; ++q) {
                tot += sAcc[q];
                if (sDiv[q] && !any) { any = true; sign = sSign[q]; }
            }
            seg_store(out, out_f64, i, seg_finish(tot, any, sign, c.functional, apply_root, p_));
        }
        __syncthreads();
    }
}

cudaError_t launch_segments(const pcf_csr* x, int functional, double p, int apply_root,
                            double lo, double hi, int precision, void* out, int out_f64,
                            Header* hdr, int32_t* long_list, cudaStream_t s)
{
    if (x->n == 0) return cudaSuccess;
    int64_t blocks = (x->n * 32 + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    const int long_blocks = device_sm_count() * 4;
    const bool f32 = precision != PCF_PREC_F64;
    const int fn = functional == PCF_FN_INTEGRAL ? kFnIntegral
                   : p == 1.0 ? kFnAbs : p == 2.0 ? kFnSquare : p == 3.0 ? kFnCube : kFnPow;
#define PCF_SEG_FN(TIN, TW, FN)                                                                   \
    {                                                                                             \
        segment_kernel<TIN, TW, FN><<<(int)blocks, 256, 0, s>>>(x->offsets, c, x->n, x->nnz,      \
                                                                apply_root, p, out, out_f64,      \
                                                                long_list);                       \
        segment_long_kernel<TIN, TW, FN><<<long_blocks, 256, 0, s>>>(x->offsets, c, apply_root,   \
                                                                     p, out, out_f64, long_list); \
    }
#define PCF_SEG_LAUNCH(TIN, TW)                                                                   \
    {                                                                                             \
        SegCtx<TIN, TW> c{(const TIN*)x->times, (const TIN*)x->values, functional, (TW)p, (TW)lo, \
                          (TW)hi, hdr, sizeof(TIN) == 8 && sizeof(TW) == 4,                       \
                          lo > 0.0 || !std::isinf(hi)};                                           \
        switch (fn) {                                                                             \
        case kFnIntegral: PCF_SEG_FN(TIN, TW, kFnIntegral) break;                                 \
        case kFnAbs: PCF_SEG_FN(TIN, TW, kFnAbs) break;                                           \
        case kFnSquare: PCF_SEG_FN(TIN, TW, kFnSquare) break;                                     \
        case kFnCube: PCF_SEG_FN(TIN, TW, kFnCube) break;                                         \
        default: PCF_SEG_FN(TIN, TW, kFnPow) break;                                               \
        }                                                                                         \
    }
    if (x->dtype == PCF_F64) {
        if (f32) PCF_SEG_LAUNCH(double, float) else PCF_SEG_LAUNCH(double, double)
    } else {
        if (f32) PCF_SEG_LAUNCH(float, float) else PCF_SEG_LAUNCH(float, double)
    }
#undef PCF_SEG_FN
#undef PCF_SEG_LAUNCH
    return cudaGetLastError();
}

}  // namespace pcfgb
