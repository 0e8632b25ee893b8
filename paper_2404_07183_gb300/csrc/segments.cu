// segments.cu -- single-PCF functionals by segment iteration (Sec. 3.2, Alg. 3).
//
// out[i] = r( int_a^b h(f_i(t)) dt ) with h(v) = v (the integral of f) or
// h(v) = |v|^p (r = x^(1/p) when requested: the L_p norm).  A PCF's segments
// [t_k, t_{k+1}) (the last one reaching inf) are clipped to [a, b].  A last
// segment reaching b = inf adds 0 when h = 0 and h * inf otherwise.
// Arithmetic per segment: float64 (PCF_PREC_F64), or float32 with Kahan's
// compensated summation per segment (PCF_PREC_F32_COMP; float64 data are
// rounded to float32 first).
//
// GPU design: one flat, element-balanced pass over the breakpoint arrays.
//  * seg_table_kernel (thread per PCF) checks the offsets with the reasons and
//    indices of pcf_pairwise's check and writes table[c] = number of PCFs that
//    start before element c * kSegChunk, for every chunk c, flagged when that
//    PCF is long (more than kSegLong breakpoints).
//  * segment_kernel: CTA c owns the PCFs that start in chunk c (table[c] ..
//    table[c + 1] - 1) and integrates every segment of them, so the last one
//    may run past the chunk's end; no two CTAs share a PCF and no CTA waits
//    for another.  The owned elements are streamed in rounds of 256 threads
//    x 16 consecutive float elements (8 double), with 16-byte vector loads
//    when the arrays are aligned.  Each thread integrates its elements in
//    order and splits them into runs at PCF starts (a bit mask built from
//    the batch's offsets in shared memory); a CTA-wide segmented scan of the
//    runs' partial sums (warp shuffles, then every warp over the eight warp
//    totals, one barrier per round) carries a PCF's partial sum across
//    threads and rounds in a fixed order.  A finished PCF's raw integral is
//    parked in shared memory and the batch's PCFs are finished (tail rule,
//    root) and stored together at the end of the batch.
//  * A long PCF (the last of its first chunk) is left out of that pass and
//    split at the chunk edges into pieces; segment_piece_kernel, a second
//    grid that starts while segment_kernel is still running, integrates each
//    piece with one CTA, and the CTA that finishes a PCF's last piece sums
//    the pieces' Kahan pairs in piece order (no CTA waits for another).
//  * The input check of pcf_pairwise runs on the same loads (same reasons,
//    same indices; an offsets error found by the table pass stops the
//    integration, element errors leave every element checked so the smallest
//    index wins).
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

constexpr int kSegThreads = 256;
// consecutive elements per thread: 16 float (4 x 16-byte loads per array) or 8 double
template <typename Tin> __host__ __device__ constexpr int seg_items() { return sizeof(Tin) == 4 ? 16 : 8; }
// elements whose PCFs a CTA owns: 1.875 rounds of 4,096 (3.75 of 2,048), so the
// chunk plus the overflow of its last PCF usually fits 2 (4) rounds instead
// of spilling a few hundred elements into an extra round
constexpr int64_t kSegChunk = 7680;
constexpr int kSegBatch = 512;         // PCF offsets staged at a time
// PCFs longer than kSegLong breakpoints are not integrated by the CTA that
// owns them but split into pieces of kSegChunk breakpoints, one CTA each,
// whose Kahan partials a combine pass sums in piece order
constexpr int64_t kSegLong = 4 * kSegChunk;
// Chunk table entry: the PCF count in the low bits; kTabLong: the PCF before
// the boundary (index count - 1) is longer than kSegLong; kTabCover: that
// long PCF also covers the boundary's breakpoint (it ends after it).
constexpr int64_t kTabLong = 1ll << 62;
constexpr int64_t kTabCover = 1ll << 61;
constexpr int64_t kTabCount = kTabCover - 1;

// Partial integral of one piece of a long PCF: the Kahan pair (float64 form:
// s only) and the sign of an infinite last segment (0 if none).
struct SegPart { double s, c; int div; int pad; };

// Partial sum of a run of segments with the head flag of the segmented scan:
// flag = a PCF starts inside the run, so nothing before it is added.
// float64: plain sum.  float32: Kahan pair, value = s - c.
template <typename T> struct SegSum;
template <> struct SegSum<double> {
    double s;
    int flag;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double h, double len) { s = fma(h, len, s); }
    __device__ __forceinline__ double value() const { return s; }
    // sum of an earlier run a and a later run b
    __device__ __forceinline__ static SegSum join(const SegSum& a, const SegSum& b)
    {
        SegSum r;
        r.flag = a.flag | b.flag;
        r.s = b.flag ? b.s : a.s + b.s;
        return r;
    }
    __device__ __forceinline__ SegSum shfl_up(int o) const
    {
        SegSum r;
        r.s = __shfl_up_sync(0xffffffffu, s, o);
        r.flag = __shfl_up_sync(0xffffffffu, flag, o);
        return r;
    }
    __device__ __forceinline__ SegSum shfl_idx(int l) const
    {
        SegSum r;
        r.s = __shfl_sync(0xffffffffu, s, l);
        r.flag = __shfl_sync(0xffffffffu, flag, l);
        return r;
    }
    __device__ __forceinline__ SegSum shfl_down(int o) const
    {
        SegSum r;
        r.s = __shfl_down_sync(0xffffffffu, s, o);
        r.flag = __shfl_down_sync(0xffffffffu, flag, o);
        return r;
    }
    __device__ __forceinline__ void to_part(SegPart& p) const { p.s = s; p.c = 0.0; }
    __device__ __forceinline__ static SegSum from_part(const SegPart* p)
    {
        SegSum r;
        r.s = __ldcg(&p->s);
        r.flag = 0;
        return r;
    }
};
template <> struct SegSum<float> {
    float s, c;
    int flag;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    // Kahan: the term h * len is formed inside the FMA that removes the
    // running compensation, then t = s + y, c = (t - s) - y, s = t.
    __device__ __forceinline__ void add(float h, float len)
    {
        const float y = __fmaf_rn(h, len, -c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
    // (s_a - c_a) + (s_b - c_b): Knuth's TwoSum of the sums (exact: t + e),
    // the rounding error e joining the compensations.
    __device__ __forceinline__ static SegSum join(const SegSum& a, const SegSum& b)
    {
        SegSum r;
        r.flag = a.flag | b.flag;
        if (b.flag) { r.s = b.s; r.c = b.c; return r; }
        const float t = __fadd_rn(a.s, b.s);
        const float bp = __fsub_rn(t, a.s);
        const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(b.s, bp));
        r.s = t;
        r.c = __fsub_rn(__fadd_rn(a.c, b.c), e);
        return r;
    }
    __device__ __forceinline__ SegSum shfl_up(int o) const
    {
        SegSum r;
        r.s = __shfl_up_sync(0xffffffffu, s, o);
        r.c = __shfl_up_sync(0xffffffffu, c, o);
        r.flag = __shfl_up_sync(0xffffffffu, flag, o);
        return r;
    }
    __device__ __forceinline__ SegSum shfl_idx(int l) const
    {
        SegSum r;
        r.s = __shfl_sync(0xffffffffu, s, l);
        r.c = __shfl_sync(0xffffffffu, c, l);
        r.flag = __shfl_sync(0xffffffffu, flag, l);
        return r;
    }
    __device__ __forceinline__ SegSum shfl_down(int o) const
    {
        SegSum r;
        r.s = __shfl_down_sync(0xffffffffu, s, o);
        r.c = __shfl_down_sync(0xffffffffu, c, o);
        r.flag = __shfl_down_sync(0xffffffffu, flag, o);
        return r;
    }
    // a float pair is stored exactly in the float64 fields of a SegPart
    __device__ __forceinline__ void to_part(SegPart& p) const { p.s = s; p.c = c; }
    __device__ __forceinline__ static SegSum from_part(const SegPart* p)
    {
        SegSum r;
        r.s = (float)__ldcg(&p->s);
        r.c = (float)__ldcg(&p->c);
        r.flag = 0;
        return r;
    }
};

template <typename T>
__device__ __forceinline__ SegSum<T> seg_identity()
{
    SegSum<T> r;
    r.zero();
    r.flag = 0;
    return r;
}

template <typename Tin, typename T>
struct SegArgs {
    const int64_t* offsets;
    const Tin* times;
    const Tin* values;
    int64_t n, nnz;
    const int64_t* table;          // [nchunks + 1]
    int functional;
    int apply_root;
    double p;                      // exponent of the functional (float64)
    T pw, lo, hi;                  // exponent and bounds in the arithmetic type
    SegPart* part_start;           // [nchunks]: piece of the long PCF starting in chunk c
    SegPart* part_cover;           // [nchunks]: piece of the long PCF covering chunk c's start
    unsigned int* long_done;       // [nchunks]: pieces finished, by the long PCF's first chunk
    void* out;
    int out_f64;
    Header* hdr;
};

// Offsets check per PCF (the reasons and indices of pcf_pairwise's check)
// and the chunk table: table[c] = #PCFs starting before element c * chunk.
__global__ void seg_table_kernel(const int64_t* __restrict__ offsets, int64_t n, int64_t nnz,
                                 int64_t nchunks, int64_t* __restrict__ table,
                                 unsigned int* __restrict__ long_done, Header* hdr)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) table[0] = 0;
    for (int64_t c = i0; c < nchunks; c += stride) long_done[c] = 0u;   // pieces finished
    for (int64_t i = i0; i < n; i += stride) {
        const int64_t o0 = offsets[i], o1 = offsets[i + 1];
        bool bad = !(o0 >= 0 && o1 > o0 && o1 <= nnz && (o1 - o0) < (1ll << 31));
        if (i == 0 && o0 != 0) bad = true;
        if (i == n - 1 && o1 != nnz) bad = true;
        if (bad) { record_error(hdr, kErrOffsets, i); continue; }
        const int64_t lng = o1 - o0 > kSegLong ? kTabLong : 0;
        // chunks 0 < c < nchunks with o0 < c * chunk <= o1 see PCFs 0..i
        // starting before them (exactly one i per c); the last PCF writes the
        // end entry
        int64_t c1 = o1 / kSegChunk;
        if (c1 > nchunks - 1) c1 = nchunks - 1;
        for (int64_t c = o0 / kSegChunk + 1; c <= c1; ++c)
            table[c] = (i + 1) | lng | (lng && c * kSegChunk < o1 ? kTabCover : 0);
        if (i == n - 1) table[nchunks] = n | lng;
    }
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

// Elements [k0, k0 + N) of times and values.  VEC: 16-byte loads (the
// arrays are 16-byte aligned and k0 is a multiple of N).
template <typename Tin, bool VEC, int N>
__device__ __forceinline__ void seg_load(const Tin* __restrict__ times, const Tin* __restrict__ values,
                                         int64_t nnz, int64_t k0, Tin (&t)[N], Tin (&v)[N])
{
    if (VEC && k0 + N <= nnz) {
        if constexpr (sizeof(Tin) == 4) {
            const float4* pt = reinterpret_cast<const float4*>(times + k0);
            const float4* pv = reinterpret_cast<const float4*>(values + k0);
#pragma unroll
            for (int u = 0; u < N / 4; ++u) {
                const float4 a = __ldg(pt + u), b = __ldg(pv + u);
                t[4 * u] = a.x; t[4 * u + 1] = a.y; t[4 * u + 2] = a.z; t[4 * u + 3] = a.w;
                v[4 * u] = b.x; v[4 * u + 1] = b.y; v[4 * u + 2] = b.z; v[4 * u + 3] = b.w;
            }
        } else {
            const double2* pt = reinterpret_cast<const double2*>(times + k0);
            const double2* pv = reinterpret_cast<const double2*>(values + k0);
#pragma unroll
            for (int u = 0; u < N / 2; ++u) {
                const double2 a = __ldg(pt + u), b = __ldg(pv + u);
                t[2 * u] = a.x; t[2 * u + 1] = a.y;
                v[2 * u] = b.x; v[2 * u + 1] = b.y;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const bool in = k0 + q < nnz;
            t[q] = in ? __ldg(times + k0 + q) : Tin(0);
            v[q] = in ? __ldg(values + k0 + q) : Tin(0);
        }
    }
}

// The input check of one element (reasons and indices of pcf_pairwise's
// check); only run by a thread whose fast check found something wrong.
template <typename Tin, bool R32>
__device__ __noinline__ void seg_record(Header* hdr, int64_t k, Tin tk, Tin vk, Tin tp, bool is_first)
{
    if (!isfinite(tk)) { record_error(hdr, kErrTimeNaN, k); return; }
    if (!isfinite(vk)) { record_error(hdr, kErrValueNaN, k); return; }
    if (is_first) {
        if (tk != Tin(0)) record_error(hdr, kErrT0, k);
    } else if (!(tk > tp)) {
        record_error(hdr, kErrOrder, k);
    }
    if (R32 && (fabs((double)tk) > (double)FLT_MAX || fabs((double)vk) > (double)FLT_MAX))
        record_error(hdr, kErrRange32, k);
}

// Fast input check of a thread's elements, on the pipes the arithmetic does
// not saturate: it only has to notice that something may be wrong (the exact
// report is made by seg_record).  Non-finite values poison a float
// accumulator (x * 0 is NaN for inf and NaN) or, for float64 arithmetic, the
// largest exponent field seen; the widths t_{k+1} - t_k between elements of
// one PCF must stay > 0 (float compare, or the order of the bit patterns of
// float64 times, which catches the first descent below a non-negative time).
template <typename Tin, typename T>
struct SegCheck {
    float fin = 0.f, md = INFINITY;      // float data or float arithmetic
    unsigned emax = 0u;                  // float64 data, float64 arithmetic
    bool order_bad = false;
    __device__ __forceinline__ void value(Tin t, Tin v)
    {
        if constexpr (sizeof(T) == 4) fin = fmaf((float)t, 0.f, fmaf((float)v, 0.f, fin));
        else if constexpr (sizeof(Tin) == 4) fin = fmaf(t, 0.f, fmaf(v, 0.f, fin));
        else {
            const unsigned a = (unsigned)__double2hiint(t) & 0x7ff00000u;
            const unsigned b = (unsigned)__double2hiint(v) & 0x7ff00000u;
            emax = max(emax, max(a, b));
        }
    }
    // t_next > t within one PCF
    __device__ __forceinline__ void order(Tin t, Tin t_next)
    {
        if constexpr (sizeof(Tin) == 4 || sizeof(T) == 4) {
            const float d = (float)t_next - (float)t;
            md = fminf(md, d);
        } else {
            order_bad |= !(__double_as_longlong(t_next) > __double_as_longlong(t));
        }
    }
    __device__ __forceinline__ bool bad() const
    {
        return fin != 0.f || !(md > 0.f) || emax == 0x7ff00000u || order_bad;
    }
};

// Fixed-order sum of the 32 lanes' pairs into lane 0 (lane l before l + 1).
template <typename T>
__device__ __forceinline__ SegSum<T> seg_warp_sum(SegSum<T> acc)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const SegSum<T> other = acc.shfl_down(o);
        if ((lane & (2 * o - 1)) == 0) acc = SegSum<T>::join(acc, other);
    }
    return acc;
}

// Breakpoints [ks, ke) of the long PCF with breakpoints o0 .. o1 - 1,
// integrated by the whole CTA (N consecutive breakpoints per thread and
// round, the threads' Kahan pairs summed in a fixed order), with the input
// check of the main pass.  The result is valid in thread 0.
template <typename Tin, typename T, int FN, bool VEC, bool CLIP>
__device__ __forceinline__ SegPart seg_piece(const SegArgs<Tin, T>& g, int64_t o0, int64_t o1, int64_t ks,
                             int64_t ke, SegSum<T>* red, int* red_div)
{
    using Sum = SegSum<T>;
    constexpr int N = seg_items<Tin>();
    constexpr int64_t kRound = (int64_t)kSegThreads * N;
    constexpr bool R32 = sizeof(Tin) == 8 && sizeof(T) == 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Sum acc = seg_identity<T>();
    int div = 0;
    SegCheck<Tin, T> chk;
    bool bad = false;
    const int64_t rb = ks - (ks % N);
    for (int64_t k0 = rb + (int64_t)tid * N; k0 < ke; k0 += kRound) {
        Tin tt[N], vv[N];
        seg_load<Tin, VEC, N>(g.times, g.values, g.nnz, k0, tt, vv);
        const Tin t_prev = k0 > 0 ? __ldg(g.times + k0 - 1) : Tin(0);
        const Tin t_next = k0 + N < g.nnz ? __ldg(g.times + k0 + N) : Tin(INFINITY);
#pragma unroll
        for (int u = 0; u < N; ++u) {
            const int64_t k = k0 + u;
            if (k < ks || k >= ke) continue;
            const Tin tk = tt[u], vk = vv[u];
            const Tin tp = u > 0 ? tt[u - 1] : t_prev;
            const Tin tn = u + 1 < N ? tt[u + 1] : t_next;
            chk.value(tk, vk);
            if (k == o0) bad |= tk != Tin(0);
            else chk.order(tp, tk);
            const T tkT = (T)tk, tnT = (T)tn;
            const T h = seg_h<FN, T>((T)vk, g.pw);
            if (k + 1 < o1) {
                if (CLIP) {
                    const T l = tkT > g.lo ? tkT : g.lo;
                    const T rr = tnT < g.hi ? tnT : g.hi;
                    if (rr > l) acc.add(h, rr - l);
                } else {
                    acc.add(h, tnT - tkT);
                }
            } else if (CLIP) {
                // last segment [t_k, inf) clipped to [a, b]
                const T l = tkT > g.lo ? tkT : g.lo;
                if (g.hi > l) {
                    if (isinf(g.hi)) {
                        if (h != T(0)) div = h > T(0) ? 1 : -1;
                    } else {
                        acc.add(h, g.hi - l);
                    }
                }
            } else if (h != T(0)) {
                div = h > T(0) ? 1 : -1;
            }
        }
    }
    if (bad || chk.bad()) {
        // exact report, as in the main pass
        for (int64_t k0 = rb + (int64_t)tid * N; k0 < ke; k0 += kRound)
            for (int u = 0; u < N; ++u) {
                const int64_t k = k0 + u;
                if (k < ks || k >= ke) continue;
                const Tin tp = k > 0 ? __ldg(g.times + k - 1) : Tin(0);
                seg_record<Tin, R32>(g.hdr, k, __ldg(g.times + k), __ldg(g.values + k), tp, k == o0);
            }
    }
    acc = seg_warp_sum<T>(acc);
    const int wdiv = __reduce_add_sync(0xffffffffu, div);   // one thread at most holds the end
    if (lane == 0) { red[warp] = acc; red_div[warp] = wdiv; }
    __syncthreads();
    SegPart out{};
    if (tid == 0) {
        Sum tot = red[0];
        int dv = red_div[0];
        for (int w = 1; w < kSegThreads / 32; ++w) {
            tot = Sum::join(tot, red[w]);
            dv += red_div[w];
        }
        tot.to_part(out);
        out.div = dv;
    }
    __syncthreads();
    return out;
}

// Piece `slot` of the long PCF i has been integrated (result in thread 0):
// store it; the CTA that finishes the PCF's last piece sums the pieces in
// order (the piece in its first chunk, then the chunks it covers) with one
// warp, applies the tail rule and the root, and stores the result.  No CTA
// waits for another: the last one to count in does the combine.
template <typename Tin, typename T>
__device__ void seg_piece_done(const SegArgs<Tin, T>& g, int64_t i, SegPart* slot,
                               const SegPart& part, int* s_last)
{
    using Sum = SegSum<T>;
    const int64_t o0 = g.offsets[i], o1 = g.offsets[i + 1];
    const int64_t c_s = o0 / kSegChunk, c_e = (o1 - 1) / kSegChunk;
    const int npieces = (int)(c_e - c_s + 1);
    if (threadIdx.x == 0) {
        *slot = part;
        __threadfence();
        const unsigned done = atomicAdd(&g.long_done[c_s], 1u) + 1u;
        *s_last = done == (unsigned)npieces;
        __threadfence();
    }
    __syncthreads();
    if (*s_last && threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int per = (npieces + 31) / 32;
        Sum acc = seg_identity<T>();
        int dv = 0;
        for (int k = lane * per; k < npieces && k < (lane + 1) * per; ++k) {
            const SegPart* pp = k == 0 ? &g.part_start[c_s] : &g.part_cover[c_s + k];
            acc = Sum::join(acc, Sum::from_part(pp));
            dv += __ldcg(&pp->div);
        }
        acc = seg_warp_sum<T>(acc);
        dv = __reduce_add_sync(0xffffffffu, dv);
        if (lane == 0)
            seg_store(g.out, g.out_f64, i, seg_finish(acc.value(), dv != 0, (double)(dv > 0 ? 1 : -1),
                                                      g.functional, g.apply_root, g.p));
    }
    __syncthreads();
}

// The pieces of long PCFs in chunk c (owned PCFs a .. b - 1): the part of
// PCF a - 1 that covers the chunk's first breakpoint (cover) and the part of
// PCF b - 1 that starts in the chunk (start), at most two.
template <typename Tin, typename T, int FN, bool VEC, bool CLIP>
__device__ __forceinline__ void seg_long_pieces(const SegArgs<Tin, T> g, int64_t c, int64_t a, int64_t b,
                                             bool cover, bool start)
{
    __shared__ SegSum<T> red[kSegThreads / 32];
    __shared__ int red_div[kSegThreads / 32];
    __shared__ int s_last;
    const int64_t cs0 = c * kSegChunk;
    const int64_t cs1 = cs0 + kSegChunk < g.nnz ? cs0 + kSegChunk : g.nnz;
    if (cover) {
        const int64_t pc = a - 1;
        const int64_t o0 = g.offsets[pc], o1 = g.offsets[pc + 1];
        const SegPart part =
            seg_piece<Tin, T, FN, VEC, CLIP>(g, o0, o1, cs0, o1 < cs1 ? o1 : cs1, red, red_div);
        seg_piece_done<Tin, T>(g, pc, &g.part_cover[c], part, &s_last);
    }
    if (start) {
        const int64_t ps = b - 1;
        const int64_t o0 = g.offsets[ps], o1 = g.offsets[ps + 1];
        const SegPart part = seg_piece<Tin, T, FN, VEC, CLIP>(g, o0, o1, o0, cs1, red, red_div);
        seg_piece_done<Tin, T>(g, ps, &g.part_start[c], part, &s_last);
    }
}

template <typename Tin, typename T, int FN, bool VEC, bool CLIP>
__global__ void __launch_bounds__(kSegThreads, sizeof(Tin) == 4 && sizeof(T) == 4 ? 4 : 2) segment_kernel(const SegArgs<Tin, T> g)
{
    using Sum = SegSum<T>;
    constexpr int N = seg_items<Tin>();
    constexpr int64_t kRound = (int64_t)kSegThreads * N;
    constexpr bool R32 = sizeof(Tin) == 8 && sizeof(T) == 4;   // float64 data in float32
    __shared__ int64_t soff[kSegBatch + 1];
    __shared__ double sres[kSegBatch];          // raw integrals of the batch's PCFs
    __shared__ signed char sdiv[kSegBatch];     // 0, or the sign of an infinite last segment
    // scan exchange, double-buffered by round parity (one barrier per round)
    __shared__ Sum warp_tot[2][kSegThreads / 32];
    __shared__ Sum carry_sh[2];

    // an offsets error (recorded by the table pass, before this kernel) makes
    // the chunk table meaningless: nothing to integrate.  Element errors do
    // not stop the pass, so that every element is checked.
    if (__syncthreads_or(threadIdx.x == 0 && g.hdr->err < (1ull << 62))) return;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = blockIdx.x;
    const int64_t ta = g.table[c], tb = g.table[c + 1];
    int64_t a = ta & kTabCount, b = tb & kTabCount;
    if (b > g.n) b = g.n;
    if (a > b) a = b;
    // the PCF starting in this chunk, if long (necessarily its last), is left
    // to segment_piece_kernel, which may start now
    if ((tb & kTabLong) != 0 && b > a) --b;
    asm volatile("griddepcontrol.launch_dependents;");

    for (int64_t a0 = a; a0 < b; a0 += kSegBatch) {
        const int np = (int)((b - a0) < kSegBatch ? (b - a0) : kSegBatch);
        for (int j = tid; j <= np; j += kSegThreads) soff[j] = g.offsets[a0 + j];
        if (tid == 0) carry_sh[0] = seg_identity<T>();
        __syncthreads();
        const int64_t e_lo = soff[0], e_hi = soff[np];
        const int64_t r_begin = e_lo - (e_lo % N);
        const int64_t nrounds = (e_hi - r_begin + kRound - 1) / kRound;

        for (int64_t r = 0; r < nrounds; ++r) {
            const int64_t k0 = r_begin + r * kRound + (int64_t)tid * N;
            const bool active = k0 < e_hi && k0 + N > e_lo;
            Tin tt[N], vv[N];
            if (active) {
                seg_load<Tin, VEC, N>(g.times, g.values, g.nnz, k0, tt, vv);
            } else {
#pragma unroll
                for (int q = 0; q < N; ++q) { tt[q] = Tin(0); vv[q] = Tin(0); }
            }
            // neighbours: t_{k0-1} from the lane before, t_{k0+N} from the lane after
            Tin t_prev = __shfl_up_sync(0xffffffffu, tt[N - 1], 1);
            Tin t_next = __shfl_down_sync(0xffffffffu, tt[0], 1);
            if (active && lane == 0 && k0 > 0) t_prev = __ldg(g.times + k0 - 1);
            if (active && lane == 31 && k0 + N < g.nnz) t_next = __ldg(g.times + k0 + N);

            // ---- this thread's elements, in order ----
            Sum run = seg_identity<T>();        // the open run (flag: its PCF starts here)
            Sum first = seg_identity<T>();      // a continued run that ended here
            int first_j = -1;
            int first_div = 0, run_div = 0;     // 0, or the sign of an infinite last segment
            if (active) {
                const int64_t dlo = e_lo - k0, dhi = e_hi - k0;
                const int q_lo = dlo > 0 ? (int)dlo : 0;
                const int q_hi = dhi < N ? (int)dhi : N;
                // PCF (batch-local) of the first owned element: soff[j] <= k < soff[j + 1]
                const int64_t kf = k0 + q_lo;
                int lo_j = 0, hi_j = np - 1;
                while (lo_j < hi_j) {
                    const int m = (lo_j + hi_j + 1) >> 1;
                    if (soff[m] <= kf) lo_j = m; else hi_j = m - 1;
                }
                const int j0 = lo_j;
                // bit q of bnd: a PCF of the batch starts at k0 + q (the batch end
                // counts as a start), q = 0 .. N
                uint32_t bnd = 0;
                for (int jj = j0; jj <= np; ++jj) {
                    const int64_t d = soff[jj] - k0;
                    if (d > N) break;
                    if (d >= 0) bnd |= 1u << (int)d;
                }
                const uint32_t inm = ((1u << q_hi) - 1u) & ~((1u << q_lo) - 1u);
                const uint32_t headm = bnd & inm;           // first elements of PCFs
                const uint32_t lastm = (bnd >> 1) & inm;    // last elements of PCFs
                // batch-local PCF of element q: jbase + popc(headm & bits 0..q)
                const int jbase = j0 - (int)((headm >> q_lo) & 1u);
                if (inm != (1u << N) - 1u) {
                    // edge of the owned range: the elements outside it belong to other
                    // CTAs; stand-ins (increasing finite times, value 0) add nothing
                    // and pass the check
                    if (q_lo > 0) t_prev = Tin(-2 * N);
                    if (q_hi < N) t_next = Tin(2 * N);
#pragma unroll
                    for (int q = 0; q < N; ++q) {
                        if (q < q_lo) { tt[q] = Tin(q - N); vv[q] = Tin(0); }
                        if (q >= q_hi) { tt[q] = Tin(q + 1); vv[q] = Tin(0); }
                    }
                }
                SegCheck<Tin, T> chk;
                bool bad = false;
                if (!(headm & 1u)) chk.order(t_prev, tt[0]);
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    const Tin tk = tt[q], vk = vv[q];
                    const Tin tn = q + 1 < N ? tt[q + 1] : t_next;
                    const T tkT = (T)tk, vkT = (T)vk, tnT = (T)tn;
                    chk.value(tk, vk);
                    if ((headm >> q) & 1u) {
                        bad |= tk != Tin(0);
                        run = seg_identity<T>();
                        run.flag = 1;
                        run_div = 0;
                    }
                    const T h = seg_h<FN, T>(vkT, g.pw);
                    if (!((lastm >> q) & 1u)) {
                        const T len = tnT - tkT;
                        chk.order(tk, tn);
                        if (CLIP) {
                            const T l = tkT > g.lo ? tkT : g.lo;
                            const T rr = tnT < g.hi ? tnT : g.hi;
                            if (rr > l) run.add(h, rr - l);
                        } else {
                            run.add(h, len);
                        }
                    } else {
                        // last segment [t_k, inf) clipped to [a, b]
                        if (CLIP) {
                            const T l = tkT > g.lo ? tkT : g.lo;
                            if (g.hi > l) {
                                if (isinf(g.hi)) {
                                    if (h != T(0)) run_div = h > T(0) ? 1 : -1;
                                } else {
                                    run.add(h, g.hi - l);
                                }
                            }
                        } else if (h != T(0)) {
                            run_div = h > T(0) ? 1 : -1;
                        }
                        const int j = jbase + __popc(headm & ((2u << q) - 1u));
                        if (run.flag) {
                            // the whole PCF lies in this thread's elements
                            sres[j] = run.value();
                            sdiv[j] = (signed char)run_div;
                        } else {
                            // continued from earlier threads: finished after the scan
                            first = run;
                            first_j = j;
                            first_div = run_div;
                        }
                    }
                }
                bad |= chk.bad();
                if (bad) {
                    // exact report: walk the elements again with the full check
                    // (compile-time indices keep tt / vv in registers)
#pragma unroll
                    for (int q = 0; q < N; ++q) {
                        if (q < q_lo || q >= q_hi) continue;
                        const Tin tp = q > 0 ? tt[q - 1] : t_prev;
                        seg_record<Tin, R32>(g.hdr, k0 + q, tt[q], vv[q], tp,
                                             ((headm >> q) & 1u) != 0);
                    }
                }
                // a PCF starts in this thread: nothing before it is carried on
                run.flag = headm != 0u ? 1 : 0;
            }

            // ---- segmented scan of the open runs: carry into each thread ----
            const int par = (int)(r & 1);
            Sum inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Sum up = inc.shfl_up(o);
                if (lane >= o) inc = Sum::join(up, inc);
            }
            Sum exc = inc.shfl_up(1);
            if (lane == 0) exc = seg_identity<T>();
            if (lane == 31) warp_tot[par][warp] = inc;
            __syncthreads();
            // every warp scans the warp totals before its own (and the carry of
            // the rounds before); the last warp publishes the next carry
            {
                const Sum cin = carry_sh[par];
                Sum winc = lane < warp ? warp_tot[par][lane] : seg_identity<T>();
#pragma unroll
                for (int o = 1; o < kSegThreads / 32; o <<= 1) {
                    const Sum up = winc.shfl_up(o);
                    if (lane >= o) winc = Sum::join(up, winc);
                }
                // lane warp - 1 now holds warps 0 .. warp-1 combined
                Sum before = winc.shfl_idx(warp > 0 ? warp - 1 : 0);
                if (warp == 0) before = seg_identity<T>();
                const Sum pre = Sum::join(cin, before);
                if (warp == kSegThreads / 32 - 1 && lane == 31)
                    carry_sh[par ^ 1] = Sum::join(pre, inc);
                if (first_j >= 0) {
                    const Sum tot = Sum::join(Sum::join(pre, exc), first);
                    sres[first_j] = tot.value();
                    sdiv[first_j] = (signed char)first_div;
                }
            }
        }
        __syncthreads();
        // ---- finish the batch's PCFs (tail rule, root) with coalesced stores ----
        for (int j = tid; j < np; j += kSegThreads)
            seg_store(g.out, g.out_f64, a0 + j,
                      seg_finish(sres[j], sdiv[j] != 0, (double)sdiv[j], g.functional,
                                 g.apply_root, g.p));
        __syncthreads();   // soff, sres and the carry are rewritten by the next batch
    }
}

// Long PCFs, piece by piece, in a second grid launched as a programmatic
// dependent of segment_kernel: it needs only the chunk table, so it starts
// once every segment_kernel CTA has started and runs in that kernel's tail.
// CTA k looks at chunks k, k + grid, k + 2 grid, ... (the pieces of one long
// PCF lie in consecutive chunks and so spread over the CTAs) and integrates
// the pieces of the flagged ones.  Every CTA finally waits for segment_kernel
// to complete, so this grid never completes before it.
template <typename Tin, typename T, int FN, bool VEC, bool CLIP>
__global__ void __launch_bounds__(kSegThreads, 2) segment_piece_kernel(const SegArgs<Tin, T> g,
                                                                       int64_t nchunks)
{
    __shared__ int64_t list[kSegThreads];
    __shared__ int list_n;
    if (!__syncthreads_or(threadIdx.x == 0 && g.hdr->err < (1ull << 62))) {
        const int64_t G = gridDim.x;
        for (int64_t base = blockIdx.x; base < nchunks; base += G * kSegThreads) {
            if (threadIdx.x == 0) list_n = 0;
            __syncthreads();
            const int64_t c = base + (int64_t)threadIdx.x * G;
            if (c < nchunks) {
                const int64_t ta = g.table[c], tb = g.table[c + 1];
                if ((ta & kTabCover) || ((tb & kTabLong) && (tb & kTabCount) > (ta & kTabCount)))
                    list[atomicAdd(&list_n, 1)] = c;
            }
            __syncthreads();
            const int m = list_n;
            for (int k = 0; k < m; ++k) {
                const int64_t cc = list[k];
                const int64_t ta = g.table[cc], tb = g.table[cc + 1];
                const int64_t a = ta & kTabCount, b = tb & kTabCount;
                seg_long_pieces<Tin, T, FN, VEC, CLIP>(g, cc, a, b, (ta & kTabCover) != 0,
                                                       (tb & kTabLong) != 0 && b > a);
            }
            __syncthreads();   // the list is rewritten
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

cudaError_t launch_segments(const pcf_csr* x, int functional, double p, int apply_root,
                            double lo, double hi, int precision, void* out, int out_f64,
                            Header* hdr, void* scratch, cudaStream_t s)
{
    if (x->n == 0) return cudaSuccess;
    const int64_t nchunks = (x->nnz + kSegChunk - 1) / kSegChunk;
    // scratch: chunk table [nchunks + 1], the two piece arrays [nchunks] and
    // the pieces-finished counters [nchunks]: 60 bytes per chunk of 7,680
    // breakpoints (+ 8), within the 16 bytes per breakpoint (256 at least)
    // the call's workspace provides
    char* sp = reinterpret_cast<char*>(scratch);
    int64_t* table = reinterpret_cast<int64_t*>(sp);
    SegPart* part_start = reinterpret_cast<SegPart*>(sp + 8 * (nchunks + 1));
    SegPart* part_cover = part_start + nchunks;
    unsigned int* long_done = reinterpret_cast<unsigned int*>(part_cover + nchunks);
    {
        int64_t blocks = ((x->n > nchunks ? x->n : nchunks) + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 16;
        if (blocks > cap) blocks = cap;
        seg_table_kernel<<<(int)blocks, 256, 0, s>>>(x->offsets, x->n, x->nnz, nchunks, table,
                                                      long_done, hdr);
    }
    if (nchunks == 0) return cudaGetLastError();
    const bool f32 = precision != PCF_PREC_F64;
    const int fn = functional == PCF_FN_INTEGRAL ? kFnIntegral
                   : p == 1.0 ? kFnAbs : p == 2.0 ? kFnSquare : p == 3.0 ? kFnCube : kFnPow;
    const bool vec = ((uintptr_t)x->times % 16 == 0) && ((uintptr_t)x->values % 16 == 0);
    const bool clip = lo > 0.0 || !std::isinf(hi);
    // a PCF longer than kSegLong needs more than kSegLong breakpoints in all
    const bool long_possible = x->nnz > kSegLong;
    const unsigned pgrid =
        (unsigned)(nchunks < 2 * (int64_t)device_sm_count() ? nchunks : 2 * device_sm_count());
    cudaError_t e = cudaSuccess;
    // programmatic dependent launch: the piece grid may start before
    // segment_kernel completes (it reads nothing segment_kernel writes)
    auto launch_pieces = [&](auto kernel, const auto& g) {
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(pgrid);
        cfg.blockDim = dim3(kSegThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, g, nchunks);
    };
#define PCF_SEG_GO(TIN, TW, FN)                                                                    \
    {                                                                                              \
        SegArgs<TIN, TW> g{x->offsets, (const TIN*)x->times, (const TIN*)x->values, x->n, x->nnz,  \
                           table, functional, apply_root ? 1 : 0, p, (TW)p, (TW)lo, (TW)hi,        \
                           part_start, part_cover, long_done, out, out_f64, hdr};                  \
        const unsigned grid = (unsigned)nchunks;                                                   \
        if (vec && clip) segment_kernel<TIN, TW, FN, true, true><<<grid, kSegThreads, 0, s>>>(g);  \
        else if (vec) segment_kernel<TIN, TW, FN, true, false><<<grid, kSegThreads, 0, s>>>(g);    \
        else if (clip) segment_kernel<TIN, TW, FN, false, true><<<grid, kSegThreads, 0, s>>>(g);   \
        else segment_kernel<TIN, TW, FN, false, false><<<grid, kSegThreads, 0, s>>>(g);            \
        if (long_possible) {                                                                        \
            if (vec && clip) e = launch_pieces(segment_piece_kernel<TIN, TW, FN, true, true>, g);   \
            else if (vec) e = launch_pieces(segment_piece_kernel<TIN, TW, FN, true, false>, g);     \
            else if (clip) e = launch_pieces(segment_piece_kernel<TIN, TW, FN, false, true>, g);    \
            else e = launch_pieces(segment_piece_kernel<TIN, TW, FN, false, false>, g);             \
        }                                                                                           \
    }
#define PCF_SEG_LAUNCH(TIN, TW)                                                                    \
    switch (fn) {                                                                                  \
    case kFnIntegral: PCF_SEG_GO(TIN, TW, kFnIntegral) break;                                      \
    case kFnAbs: PCF_SEG_GO(TIN, TW, kFnAbs) break;                                                \
    case kFnSquare: PCF_SEG_GO(TIN, TW, kFnSquare) break;                                          \
    case kFnCube: PCF_SEG_GO(TIN, TW, kFnCube) break;                                              \
    default: PCF_SEG_GO(TIN, TW, kFnPow) break;                                                    \
    }
    if (x->dtype == PCF_F64) {
        if (f32) PCF_SEG_LAUNCH(double, float) else PCF_SEG_LAUNCH(double, double)
    } else {
        if (f32) PCF_SEG_LAUNCH(float, float) else PCF_SEG_LAUNCH(float, double)
    }
#undef PCF_SEG_GO
#undef PCF_SEG_LAUNCH
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace pcfgb
