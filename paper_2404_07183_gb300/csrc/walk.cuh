// walk.cuh -- persistent pair-tile merge walk (rectangle iteration, Sec. 3
// Alg. 1, with the accumulation of Alg. 2 / Eq. simpleint fused in).
//
// Work decomposition
//   * PCFs are sorted by length and cut into blocks of 32; a tile is a
//     (row block, column block) pair: 32 x 32 = 1024 pairs.  Pairwise calls
//     visit the upper triangle of blocks; cross calls all blocks.  Tiles are
//     handed out by one atomic counter (longest PCFs first) to one persistent
//     1024-thread CTA per SM.
//   * Warp w of the CTA takes the tile's w-th diagonal: lane l walks the pair
//     (row (l + w) mod 32, column l).  Every lane of a half-warp (quarter-warp
//     for 16-byte elements) therefore reads a different PCF of each side.
//   * The tile's 64 PCFs are staged in shared memory in four regions of 16
//     PCFs; element k of PCF slot s sits at (k * 16 + s) * sizeof(element), so
//     the 16 PCFs of a region fall into 16 different bank groups and the
//     data-dependent reads of a warp are free of bank conflicts whatever
//     positions the lanes have reached.
//   * Long PCFs are staged in time windows [T0, T1): T1 is the smallest end
//     time of the W-th remaining element over the tile's PCFs, so every PCF's
//     elements up to T1 fit (keyed and float64 walks may give the row side
//     more of the window memory than the column side, or less, each window:
//     see the split below).  A lane walks exactly the rectangles that end
//     before T1 and resumes in the next window at element 0 of both its PCFs;
//     the rectangles, their order and their arithmetic are the same as in one
//     uninterrupted walk.
//
// The merge step (one rectangle per step, one side advances per step).
// A lane holds, for each of its PCFs f (row) and g (column), the current
// interval element (end time te, value v) and its shared-memory offset.  A
// step emits the rectangle [tc, min(te_f, te_g)) with value h(v_f, v_g) and
// then loads the next element of the side whose interval ends first (f on a
// tie).  The two loads are predicated per lane: f-loads only touch the row
// regions and g-loads only the column regions, so each stays bank-conflict
// free.  A breakpoint shared by both PCFs costs one extra step whose rectangle
// has width 0 (h * 0 = 0 added to the accumulator).  The step count of a pair
// is n_f + n_g - 2 plus the tail, known before the walk starts.
//
// Keyed form (KEYED = 1: float64 input walked in float32).  Interval elements
// are KElem: the end time's exact order key (its rank among the call's
// interval ends, keys.cu), the end time as float32 hi + lo, and the value.
// The advancing side is chosen by one unsigned compare of the keys, so every
// comparison is decided on the float64 times, and a rectangle's width is
// (hi_n - hi_c) + (lo_n - lo_c): hi_n - hi_c is exact when the hi parts are
// within a factor 2 of each other (Sterbenz) and the lo parts carry the rest
// of the float64 difference, so the width is within about u * w + 2^-48 * t
// of the exact one (hi + lo holds about 48 bits of t) instead of u * t.
#pragma once

#include <cmath>

#include "internal.cuh"

namespace pcfgb {

constexpr int kF64 = 0, kF32C = 1, kF32 = 2, kF32B = 3;
constexpr int MI_NONE = 0, MI_L1 = 1, MI_L2 = 2, MI_L3 = 3, MI_LP = 4, MI_GRAM = 5;

__host__ __device__ constexpr int combo_n(int c)
{
    return (c == kComboL1L2Gram || c == kComboL1L2L3) ? 3 : 1;
}

__host__ __device__ constexpr int combo_metric(int c, int slot)
{
    return c == kComboL1 ? MI_L1
         : c == kComboL2 ? MI_L2
         : c == kComboGram ? MI_GRAM
         : c == kComboLP ? MI_LP
         : c == kComboL3 ? MI_L3
         : c == kComboL1L2Gram ? (slot == 0 ? MI_L1 : slot == 1 ? MI_L2 : MI_GRAM)
         : (slot == 0 ? MI_L1 : slot == 1 ? MI_L2 : MI_L3);
}

template <typename T> struct ElemOf;
template <> struct ElemOf<float> { using type = float2; };
template <> struct ElemOf<double> { using type = double2; };

// Element type, order-key type and accessors of a walk form.
template <typename T, bool KEYED> struct WalkForm {
    using E = typename ElemOf<T>::type;
    using K = T;                 // interval ends are compared as values
    static __device__ __forceinline__ K key(const E& e) { return e.x; }
    static __device__ __forceinline__ T val(const E& e) { return e.y; }
};
template <> struct WalkForm<float, true> {
    using E = KElem;
    using K = uint32_t;          // interval ends are compared by their order keys
    static __device__ __forceinline__ K key(const E& e) { return e.k; }
    static __device__ __forceinline__ float val(const E& e) { return e.v; }
};

// h(a, b) of Sec. 2.2 for one metric, in the walk type.
template <int MI, typename T>
__device__ __forceinline__ T term_h(T a, T b, T d, T p)
{
    if constexpr (MI == MI_L1) return fabs(d);
    else if constexpr (MI == MI_L2) return d * d;
    else if constexpr (MI == MI_L3) { T ad = fabs(d); return ad * ad * ad; }
    else if constexpr (MI == MI_LP) return pow(fabs(d), p);
    else return a * b;
}

template <int PREC> struct Acc;
template <> struct Acc<kF64> {
    double s = 0.0;
    __device__ __forceinline__ void add(double h, double dt) { s = fma(h, dt, s); }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<kF32> {
    float s = 0.f;
    __device__ __forceinline__ void add(float h, float dt) { s = fmaf(h, dt, s); }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double value() const { return (double)s; }
};
// Kahan's compensated summation, one rectangle term per add.  The term
// h * dt is formed inside the fused multiply-add that also removes the
// running compensation (y = h*dt - c, one rounding), then
//   t = s + y;  c = (t - s) - y;  s = t,
// so c holds (the negative of) the low-order part lost by each addition and
// the sum is s - c.  Error <= 2u * sum |terms| + O(n u^2).
template <> struct Acc<kF32C> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float h, float dt)
    {
        const float y = __fmaf_rn(h, dt, -c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Block-compensated float32: the rectangle terms are summed by FMA into a
// float32 partial over a block of at most 16 rectangles (one unrolled body
// of the walk loop, or the loop's remainder), and each block partial is
// added into a Kahan (sum, compensation) pair.  A block of k terms adds at
// most k*u*sum|terms| to the error, the Kahan stage 2u*sum|blocks|, so the
// total stays below about 18u * sum|terms| (1.1e-6 relative for the L_p
// integrands) at a quarter of the per-rectangle compensation work.
template <> struct Acc<kF32B> {
    float part = 0.f, s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float h, float dt) { part = fmaf(h, dt, part); }
    __device__ __forceinline__ void flush()
    {
        const float y = __fsub_rn(part, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
        part = 0.f;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int COMBO, int PREC, typename T>
__device__ __forceinline__ void accumulate(Acc<PREC>* acc, T a, T b, T dt, T p)
{
    const T d = a - b;
    acc[0].add(term_h<combo_metric(COMBO, 0)>(a, b, d, p), dt);
    if constexpr (combo_n(COMBO) > 1) acc[1].add(term_h<combo_metric(COMBO, 1)>(a, b, d, p), dt);
    if constexpr (combo_n(COMBO) > 2) acc[2].add(term_h<combo_metric(COMBO, 2)>(a, b, d, p), dt);
}

// Accumulators of one walk.  The generic form keeps one Acc per metric.
template <int PREC, int COMBO>
struct AccSet {
    static constexpr int NM = combo_n(COMBO);
    Acc<PREC> a[NM];
    template <typename T>
    __device__ __forceinline__ void add(T va, T vb, T dt, T p) { accumulate<COMBO, PREC>(a, va, vb, dt, p); }
    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int m = 0; m < NM; ++m) a[m].flush();
    }
    __device__ __forceinline__ double value(int m) const { return a[m].value(); }
    // the step's integrand values h(va, vb) per metric, before the advance
    struct Terms { float h[NM]; };
    template <typename T>
    __device__ __forceinline__ Terms terms(T va, T vb, T p) const
    {
        Terms t;
        const T d = va - vb;
        t.h[0] = term_h<combo_metric(COMBO, 0)>(va, vb, d, p);
        if constexpr (NM > 1) t.h[1] = term_h<combo_metric(COMBO, 1)>(va, vb, d, p);
        if constexpr (NM > 2) t.h[2] = term_h<combo_metric(COMBO, 2)>(va, vb, d, p);
        return t;
    }
    __device__ __forceinline__ void add_terms(const Terms& t, float dt)
    {
#pragma unroll
        for (int m = 0; m < NM; ++m) a[m].add(t.h[m], dt);
    }
};

template <int PREC, int COMBO>
struct AccFor { using type = AccSet<PREC, COMBO>; };

// Exact "x ends after y" for interval ends (non-negative, +inf allowed).
// float64 compares go to the integer pipe through the bit patterns, which
// order like the values for non-negative doubles.
__device__ __forceinline__ bool ends_after(float x, float y) { return x > y; }
__device__ __forceinline__ bool ends_after(double x, double y)
{
    return __double_as_longlong(x) > __double_as_longlong(y);
}

// Predicated advance of the side whose interval ends first (f on a tie):
// its shared-memory cursor moves to the next element (kRowBytes further) and
// the element's (end time, value) is loaded in place.  Written as PTX so the
// two loads stay predicated and land directly in the cursor registers after
// the step's arithmetic has consumed the old values (the "memory" clobber
// keeps the shared-memory reads behind the staging barrier).
template <unsigned kRowBytes>
__device__ __forceinline__ void advance_cursor(unsigned& af, float& tf, float& vf,
                                               unsigned& ag, float& tg, float& vg)
{
    asm volatile("{\n\t"
                 ".reg .pred p;\n\t"
                 "setp.le.f32 p, %1, %4;\n\t"
                 "@p add.u32 %0, %0, %6;\n\t"
                 "@p ld.shared.v2.f32 {%1, %2}, [%0];\n\t"
                 "@!p add.u32 %3, %3, %6;\n\t"
                 "@!p ld.shared.v2.f32 {%4, %5}, [%3];\n\t"
                 "}"
                 : "+r"(af), "+f"(tf), "+f"(vf), "+r"(ag), "+f"(tg), "+f"(vg)
                 : "n"(kRowBytes)
                 : "memory");
}

// float64: the order test runs on the bit patterns (integer pipe).
template <unsigned kRowBytes>
__device__ __forceinline__ void advance_cursor(unsigned& af, double& tf, double& vf,
                                               unsigned& ag, double& tg, double& vg)
{
    const long long bf = __double_as_longlong(tf), bg = __double_as_longlong(tg);
    asm volatile("{\n\t"
                 ".reg .pred p;\n\t"
                 "setp.le.s64 p, %6, %7;\n\t"
                 "@p add.u32 %0, %0, %8;\n\t"
                 "@p ld.shared.v2.f64 {%1, %2}, [%0];\n\t"
                 "@!p add.u32 %3, %3, %8;\n\t"
                 "@!p ld.shared.v2.f64 {%4, %5}, [%3];\n\t"
                 "}"
                 : "+r"(af), "+d"(tf), "+d"(vf), "+r"(ag), "+d"(tg), "+d"(vg)
                 : "l"(bf), "l"(bg), "n"(kRowBytes)
                 : "memory");
}

// Keyed advance: the side whose interval ends first is the one with the
// smaller order key (f on equal keys, i.e. equal float64 times).  One
// predicate selects that side's end (hi, lo), the rectangle's right end, and
// then advances the side, loading its next KElem (key, hi, lo, value) in
// place: the compare is made once for both.
template <unsigned kRowBytes>
__device__ __forceinline__ void advance_select_keyed(unsigned& af, uint32_t& kf, float& hf,
                                                     float& lf, float& vf, unsigned& ag,
                                                     uint32_t& kg, float& hg, float& lg, float& vg,
                                                     float& hn, float& ln)
{
    asm volatile("{\n\t"
                 ".reg .pred p;\n\t"
                 "setp.le.u32 p, %1, %6;\n\t"
                 "selp.f32 %10, %2, %7, p;\n\t"
                 "selp.f32 %11, %3, %8, p;\n\t"
                 "@p add.u32 %0, %0, %12;\n\t"
                 "@p ld.shared.v4.b32 {%1, %2, %3, %4}, [%0];\n\t"
                 "@!p add.u32 %5, %5, %12;\n\t"
                 "@!p ld.shared.v4.b32 {%6, %7, %8, %9}, [%5];\n\t"
                 "}"
                 : "+r"(af), "+r"(kf), "+f"(hf), "+f"(lf), "+f"(vf),
                   "+r"(ag), "+r"(kg), "+f"(hg), "+f"(lg), "+f"(vg), "=f"(hn), "=f"(ln)
                 : "n"(kRowBytes)
                 : "memory");
}

__device__ __forceinline__ float first_end(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double first_end(double a, double b)
{
    return __double_as_longlong(a) <= __double_as_longlong(b) ? a : b;
}

__device__ __forceinline__ double finalize_root(int metric, int root, double p, double I)
{
    if (!root || metric == PCF_GRAM) return I;
    double e = metric == PCF_L1 ? 1.0 : metric == PCF_L2 ? 2.0 : p;
    if (e == 1.0) return I;
    if (e == 2.0) return sqrt(I);
    return pow(I, 1.0 / e);
}

// Integral of the weight over a rectangle [l, l + dt): dt itself (WEIGHT 0),
// or for w(t) = exp(-lambda t) the antiderivative difference W(l + dt) - W(l)
// written as exp(-lambda l) * (-expm1(-lambda dt)) / lambda (WEIGHT 1).
template <int WEIGHT>
__device__ __forceinline__ float weight_span(float l, float dt, float lam, float inv_lam)
{
    if constexpr (WEIGHT == 0) return dt;
    else return expf(-lam * l) * (-expm1f(-lam * dt)) * inv_lam;
}
template <int WEIGHT>
__device__ __forceinline__ double weight_span(double l, double dt, double lam, double inv_lam)
{
    if constexpr (WEIGHT == 0) return dt;
    else return exp(-lam * l) * (-expm1(-lam * dt)) * inv_lam;
}

// One 32-byte sector of global memory (32-byte aligned, read-only for the
// kernel's lifetime) in a single 256-bit load.
__device__ __forceinline__ void ldg_sector(const void* p, float (&r)[8])
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]),
          "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(p));
}

__device__ __forceinline__ void decode_tile(const WalkArgs& a, int64_t t, int64_t& bi, int64_t& bj)
{
    if (a.symmetric) decode_upper_tile(a.nb_r, t, a.tile_order, bi, bj);
    else decode_cross_tile(a.nb_r, a.nb_c, t, bi, bj);
}

// CTAS: resident CTAs per SM the launch is built for (1 for 1024 threads; 2 or
// 3 for 512 threads, which caps the registers at 64 or 40 per thread).
// THREADS = 1024: one CTA per SM; a work unit is a whole 32 x 32 tile and
// warp w walks its diagonal w (lane l: row (l + w) mod 32, column l).
// THREADS = 512: two CTAs per SM, each with half the shared memory; a work
// unit is half a tile, 32 rows x 16 columns (three staged regions instead of
// four, so the window stays larger), and warp w walks lane l's pair
// (row (l + w) mod 32, column l mod 16).  Both halves of a tile belong to the
// same shard.
// WEIGHT: 0 = plain integrals, 1 = integrands weighted by exp(-lambda t).
// Integration bounds [lo, hi] (WalkArgs) apply to every variant.
template <typename T, int PREC, int COMBO, int THREADS, int CTAS, int WEIGHT = 0, bool KEYED = false>
__global__ void __launch_bounds__(THREADS, CTAS) walk_kernel(const WalkArgs a)
{
    using WF = WalkForm<T, KEYED>;
    using E = typename WF::E;
    using K = typename WF::K;                       // order key of an interval end
    constexpr int NM = combo_n(COMBO);
    constexpr int TCOLS = THREADS / 32;             // columns per work unit (32 or 16)
    constexpr int UNITS = kTile / TCOLS;            // work units per 32 x 32 tile
    constexpr int NPCF = kTile + TCOLS;             // staged PCFs: 32 rows + TCOLS columns
    constexpr unsigned kRow = kGroup * sizeof(E);   // bytes between element k and k+1 of a PCF
    // steps per unrolled body: 4 for the keyed and float64 walks, 6 for the
    // plain float32 walk (measured against 2, 8 and 16: a short remainder
    // loop per window against the loop overhead per step), except for the
    // block-compensated accumulator, whose blocks are the unrolled bodies
    // (16 rectangles)
    constexpr int kUnroll = PREC == kF32B ? 16 : (KEYED || sizeof(T) == 8 ? 4 : 6);
    static_assert(THREADS == 1024 || THREADS == 512, "thread count");
    static_assert(!KEYED || sizeof(T) == 4, "keyed walks are float32 walks");

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t sS[kTilePcfs], sNext[kTilePcfs], sLen[kTilePcfs], sStaged[kTilePcfs];
    __shared__ int64_t sOff[kTilePcfs];
    // split candidates: the keyed and float64 walks (16-byte elements, half
    // the window of the plain float32 walk) choose among five; the plain
    // float32 walk keeps the even split (measured: the choice cost it 3% on
    // the stable-rank set at its larger window)
    constexpr int kSplits = (KEYED || sizeof(T) == 8) ? 5 : 1;
    constexpr bool kAdapt = kSplits > 1;
    // window end per split candidate: [0] rows' minimum, [1] columns'
    __shared__ K sT1part[2][kSplits];
    __shared__ int sSplit;                          // split of the staged windows
    __shared__ int64_t sTile;

    if (gated_off(a.gate, a.gate_want64)) return;   // the other walk of an AUTO64 call
    if (block_sees_error(a.hdr)) return;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = a.window;
    // The window memory holds NR regions of W elements per PCF: 2 regions of
    // row PCFs and RC of column PCFs.  Each window splits it between the two
    // sides (split c gives the rows Wr(c) elements, the columns Wc(c), with
    // 2 Wr + RC Wc <= NR W), taking the split whose window reaches furthest:
    // when the rows are dense in time and the columns sparse (or the other
    // way round), the dense side gets the room, and the tile needs fewer
    // windows.
    constexpr int RC = NPCF / kGroup - 2, NR = 2 + RC;
    auto split_wr = [W](int c) { return c == 0 ? W : (W * (c == 1 ? 3 : c == 2 ? 5 : c == 3 ? 2 : 6)) / 4; };
    auto split_wc = [W](int c, int wr) { return (NR * W - 2 * wr) / RC; };
    auto split_ok = [](int wr, int wc) { return wr >= 4 && wc >= 4; };
    const T p0 = (T)a.p[0];
    const unsigned smem_base = (unsigned)__cvta_generic_to_shared(smem);
    const E* packR = reinterpret_cast<const E*>(a.pack_r);
    const E* packC = reinterpret_cast<const E*>(a.pack_c);
    // bounds as order keys: the values themselves, or (keyed) the keys the
    // key sort gave a and b; [0, inf) needs no lookup (1 orders below every
    // end, kKeyInf is the key of te = +inf)
    K lo, hi;
    if constexpr (KEYED) {
        lo = a.bound_keys ? (K)a.bound_keys[0] : (K)1u;
        hi = a.bound_keys ? (K)a.bound_keys[1] : (K)kKeyInf;
    } else {
        lo = (T)a.lo;
        hi = (T)a.hi;
    }
    // the walk closes at hi (no tail rule) when hi is finite or the weight
    // makes the last rectangle [t_last, inf) finite: exp(-lam t_last) / lam
    bool bounded;
    if constexpr (KEYED) bounded = !isinf(a.hi) || WEIGHT != 0;
    else bounded = hi < T(INFINITY) || WEIGHT != 0;
    const T lam = (T)a.lambda, inv_lam = WEIGHT ? T(1) / (T)a.lambda : T(0);
    const K k_start = lo;                           // key of the walk's first time

    // this lane's pair inside every work unit
    const int my_r = (lane + warp) & 31;
    const int my_c = lane & (TCOLS - 1);
    const int pf = my_r, pg = kTile + my_c;        // staged PCF indices
    // byte offset of staged PCF p's slot when the rows hold wr elements per
    // PCF and the columns wc (regions 0, 1: rows; 2 ..: columns)
    auto slot_base = [](int p, int wr, int wc) -> unsigned {
        const int r = p >> 4;
        const unsigned e = r < 2 ? (unsigned)r * (unsigned)wr
                                 : 2u * (unsigned)wr + (unsigned)(r - 2) * (unsigned)wc;
        return e * kRow + (unsigned)(p & 15) * (unsigned)sizeof(E);
    };
    // the even split's slots (the only ones of the plain float32 walk)
    const unsigned regionBytes = (unsigned)W * kRow;    // a region of the even split
    const unsigned even_base_f = (unsigned)(pf >> 4) * regionBytes + (unsigned)(pf & 15) * sizeof(E);
    const unsigned even_base_g = (unsigned)(pg >> 4) * regionBytes + (unsigned)(pg & 15) * sizeof(E);

    for (;;) {
        if (tid == 0) {
            const int64_t k = (int64_t)atomicAdd(&a.hdr->tiles, 1ull);
            sTile = (a.shard_index + (k / UNITS) * a.shard_count) * UNITS + (k % UNITS);
        }
        __syncthreads();
        const int64_t unit = sTile;
        const int64_t t = unit / UNITS;
        if (t >= a.ntiles) break;
        const int half = (int)(unit - t * UNITS);
        int64_t bi, bj;
        decode_tile(a, t, bi, bj);
        const int64_t col0 = bj * kTile + half * TCOLS;   // first column of this unit

        // unit metadata
        if (tid < NPCF) {
            const bool is_row = tid < kTile;
            const int64_t g = is_row ? bi * kTile + tid : col0 + (tid - kTile);
            const int64_t nset = is_row ? a.n_r : a.n_c;
            if (g < nset) {
                sLen[tid] = is_row ? a.slen_r[g] : a.slen_c[g];
                sOff[tid] = is_row ? a.poff_r[g] : a.poff_c[g];
            } else {
                sLen[tid] = 0;   // no PCF: never staged, never walked
                sOff[tid] = 0;
            }
            int start = 0;
            if (a.lo > 0.0 && sLen[tid] > 0) {
                // first element whose interval ends at or after lo
                const E* src = (is_row ? packR : packC) + sOff[tid];
                int l = 0, h = sLen[tid] - 1;
                while (l < h) {
                    const int m = (l + h) >> 1;
                    if (WF::key(src[m]) < lo) l = m + 1; else h = m;
                }
                start = l;
            }
            sS[tid] = start;
            sNext[tid] = 0;
            sStaged[tid] = -1;   // window start of what is in shared memory
        }
        if (kAdapt && tid == 0) sSplit = -1;
        const bool lane_valid = (bi * kTile + my_r < a.n_r) && (col0 + my_c < a.n_c);

        typename AccFor<PREC, COMBO>::type acc;
        // the current time tc: a value, or (keyed) float32 hi + lo
        T tc = T(0), tcl = T(0);
        if constexpr (KEYED) { tc = a.lo_hl[0]; tcl = a.lo_hl[1]; }
        else tc = (T)a.lo;
        K T0 = k_start;         // start of the current window (block-uniform)
        __syncthreads();

        for (bool first = true;; first = false) {
            // ---- advance the window starts; window end T1 = min over PCFs of
            //      te[S + W_p - 1] (clamped to the last element), W_p the
            //      share of the PCF's side (W for the even split); warp 0
            //      holds the 32 row PCFs, warp 1 the column PCFs ----
            if (!kAdapt && tid < 64) {
                // one split: the window end of the even layout
                K cand;
                if constexpr (KEYED) cand = (K)kKeyInf; else cand = T(INFINITY);
                const int len = tid < NPCF ? sLen[tid] : 0;
                if (len > 0) {
                    if (!first) sS[tid] = sNext[tid];
                    int idx = sS[tid] + W - 1;
                    if (idx > len - 1) idx = len - 1;
                    cand = WF::key((tid < kTile ? packR : packC)[sOff[tid] + idx]);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    K other = __shfl_xor_sync(0xffffffffu, cand, o);
                    cand = other < cand ? other : cand;
                }
                if (lane == 0) sT1part[warp][0] = cand;
            }
            if (kAdapt && tid < 64) {
                K kinf;
                if constexpr (KEYED) kinf = (K)kKeyInf; else kinf = T(INFINITY);
                const int len = tid < NPCF ? sLen[tid] : 0;
                if (len > 0 && !first) sS[tid] = sNext[tid];
                const int S = len > 0 ? sS[tid] : 0;
                const E* src = (tid < kTile ? packR : packC) + (len > 0 ? sOff[tid] : 0);
#pragma unroll
                for (int c = 0; c < kSplits; ++c) {
                    const int wr = split_wr(c), wc = split_wc(c, wr);
                    K cand = kinf;
                    if (len > 0 && split_ok(wr, wc)) {
                        int idx = S + (tid < kTile ? wr : wc) - 1;
                        if (idx > len - 1) idx = len - 1;
                        cand = WF::key(src[idx]);
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        K other = __shfl_xor_sync(0xffffffffu, cand, o);
                        cand = other < cand ? other : cand;
                    }
                    if (lane == 0) sT1part[warp][c] = cand;
                }
            }
            __syncthreads();
            // the split whose window reaches furthest (the even split on ties)
            int split = 0;
            K T1 = sT1part[0][0] < sT1part[1][0] ? sT1part[0][0] : sT1part[1][0];
#pragma unroll
            for (int c = 1; c < kSplits; ++c) {
                const int wr = split_wr(c), wc = split_wc(c, wr);
                const K t = sT1part[0][c] < sT1part[1][c] ? sT1part[0][c] : sT1part[1][c];
                if (split_ok(wr, wc) && t > T1 && T1 < hi) { T1 = t; split = c; }
            }
            if (T1 > hi) T1 = hi;
            const int Wr = kAdapt ? split_wr(split) : W;
            const int Wc = kAdapt ? split_wc(split, Wr) : W;
            const bool moved = kAdapt && split != sSplit;   // regions moved: stage every PCF
            // byte offset of region r (rows: 0, 1; columns: 2 ..)
            auto region_base = [&](int r) -> unsigned {
                if constexpr (!kAdapt) return (unsigned)r * regionBytes;
                return r < 2 ? (unsigned)r * (unsigned)Wr * kRow
                             : (2u * (unsigned)Wr + (unsigned)(r - 2) * (unsigned)Wc) * kRow;
            };
            auto pcf_w = [&](int p) {
                if constexpr (!kAdapt) return W;
                return p < kTile ? Wr : Wc;
            };
            const bool last = !(T1 < hi);
            if (!(T1 > T0)) {
                // more than W coincident interval ends in one PCF (only possible
                // when float64 times were rounded to float32): no progress
                if (tid == 0) record_error(a.hdr, kErrDense32, bi * kTile);
                return;
            }

            // ---- stage elements [S, S + min(W_p, len - S)) of the PCFs whose
            //      window start moved, or all of them when the split changed
            //      (the others are still in place) ----
            // THREADS is a multiple of 16, so a thread always serves the same
            // slot (tid & 15) of each region.  A thread copies whole 32-byte
            // sectors of its PCF (G elements, one 256-bit load; the packed
            // arrays are 256-byte aligned, so a sector holding one element of
            // the set lies inside its buffer) and stores the ones inside the
            // window; the 16 lanes of a half-warp store 16 different slots, so
            // the shared-memory stores are free of bank conflicts.
            {
                constexpr int G = 32 / (int)sizeof(E);
                const int slot = tid & 15;
#pragma unroll 1
                for (int region = 0; region < NPCF / kGroup; ++region) {
                    const int p = region * kGroup + slot;
                    const int S = sS[p];
                    if (S == sStaged[p] && !moved) continue;
                    const int len = sLen[p];
                    int kend = len - S;
                    if (kend > pcf_w(p)) kend = pcf_w(p);
                    const int64_t g0 = sOff[p] + S;               // first element of the window
                    const int lead = (int)(g0 & (G - 1));         // its place in its sector
                    const E* src = (p < kTile ? packR : packC) + (g0 - lead);
                    const int nsec = (kend + lead + G - 1) / G;
                    unsigned char* dst = smem + region_base(region) + (unsigned)slot * sizeof(E);
                    auto copy_sector = [&](int sc) {
                        union { float f[8]; E e[G]; } u;
                        ldg_sector(src + sc * G, u.f);
#pragma unroll
                        for (int v = 0; v < G; ++v) {
                            const int k = sc * G - lead + v;
                            if (k >= 0 && k < kend)
                                *reinterpret_cast<E*>(dst + (unsigned)k * kRow) = u.e[v];
                        }
                    };
                    if constexpr (CTAS >= 3) {
                        // 40 registers per thread: one sector in flight
                        for (int sc = tid >> 4; sc < nsec; sc += THREADS / 16) copy_sector(sc);
                    } else {
                        // up to four sectors' loads in flight per thread
#pragma unroll 4
                        for (int sc = tid >> 4; sc < nsec; sc += THREADS / 16) copy_sector(sc);
                    }
                }
            }
            __syncthreads();

            // ---- per PCF: first staged element whose interval ends at/after T1 ----
            if (tid < NPCF) {
                const int len = sLen[tid];
                int next = 0;
                if (len > 0) {
                    int cnt = len - sS[tid];
                    if (cnt > pcf_w(tid)) cnt = pcf_w(tid);
                    const unsigned colbase = region_base(tid >> 4) + (unsigned)(tid & 15) * sizeof(E);
                    int lo2 = 0, hi2 = cnt - 1;        // te[hi2] >= T1 holds by the choice of T1
                    while (lo2 < hi2) {
                        int mid = (lo2 + hi2) >> 1;
                        const K te = WF::key(*reinterpret_cast<const E*>(smem + colbase + (unsigned)mid * kRow));
                        if (te < T1) lo2 = mid + 1; else hi2 = mid;
                    }
                    next = sS[tid] + lo2;
                }
                sNext[tid] = next;
                sStaged[tid] = sS[tid];
            }
            __syncthreads();
            if (kAdapt && tid == 0) sSplit = split;

            // ---- walk this window ----
            if (lane_valid) {
                int cnt = (sNext[pf] - sS[pf]) + (sNext[pg] - sS[pg]);
                const unsigned base_f = kAdapt ? slot_base(pf, Wr, Wc) : even_base_f;
                const unsigned base_g = kAdapt ? slot_base(pg, Wr, Wc) : even_base_g;
                unsigned af = smem_base + base_f, ag = smem_base + base_g;
                const E ef = *reinterpret_cast<const E*>(smem + base_f);
                const E eg = *reinterpret_cast<const E*>(smem + base_g);
                if constexpr (KEYED) {
                    uint32_t kf = ef.k, kg = eg.k;
                    float hf = ef.hi, lf = ef.lo, vf = ef.v;
                    float hg = eg.hi, lg = eg.lo, vg = eg.v;
                    // width of [tc, te_n) from the hi and lo parts of both ends
#define PCF_WALK_STEP()                                                           \
                    {                                                             \
                        /* integrand values from the current elements, then the */ \
                        /* end of the rectangle and the advance in one PTX block */ \
                        const float va = vf, vb = vg;                             \
                        float hn, ln;                                             \
                        auto terms = acc.terms(va, vb, p0);                       \
                        advance_select_keyed<kRow>(af, kf, hf, lf, vf, ag, kg, hg, lg, vg, hn, ln); \
                        const float w = __fadd_rn(__fsub_rn(hn, tc), __fsub_rn(ln, tcl)); \
                        const float dt = weight_span<WEIGHT>(tc, w, lam, inv_lam); \
                        tc = hn;                                                  \
                        tcl = ln;                                                 \
                        acc.add_terms(terms, dt);                                 \
                    }
#pragma unroll 1
                    for (; cnt >= kUnroll; cnt -= kUnroll) {
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) PCF_WALK_STEP()
                        acc.flush();
                    }
#pragma unroll 1
                    for (; cnt > 0; --cnt) PCF_WALK_STEP()
#undef PCF_WALK_STEP
                    if (last && bounded) {
                        // closing rectangle [tc, hi) with the values holding at hi
                        const float w = __fadd_rn(__fsub_rn(a.hi_hl[0], tc), __fsub_rn(a.hi_hl[1], tcl));
                        acc.add(vf, vg, weight_span<WEIGHT>(tc, w, lam, inv_lam), p0);
                        tc = a.hi_hl[0];
                        tcl = a.hi_hl[1];
                    }
                } else {
                    T tf = ef.x, tg = eg.x, vf = ef.y, vg = eg.y;
#define PCF_WALK_STEP()                                                           \
                    {                                                             \
                        const T tn = first_end(tf, tg);                           \
                        const T dt = weight_span<WEIGHT>(tc, tn - tc, lam, inv_lam); \
                        tc = tn;                                                  \
                        acc.add(vf, vg, dt, p0);                                  \
                        advance_cursor<kRow>(af, tf, vf, ag, tg, vg);             \
                    }
#pragma unroll 1
                    for (; cnt >= kUnroll; cnt -= kUnroll) {
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) PCF_WALK_STEP()
                        acc.flush();
                    }
#pragma unroll 1
                    for (; cnt > 0; --cnt) PCF_WALK_STEP()
#undef PCF_WALK_STEP
                    if (last && bounded) {
                        // closing rectangle [tc, hi) with the values holding at hi
                        acc.add(vf, vg, weight_span<WEIGHT>(tc, hi - tc, lam, inv_lam), p0);
                        tc = hi;
                    }
                }
                acc.flush();
            }
            __syncthreads();
            if (last) break;
            T0 = T1;
        }

        // ---- tail, root, output ----
        if (lane_valid) {
            const int64_t gi = bi * kTile + my_r, gj = col0 + my_c;
            const int64_t i = a.perm_r[gi], j = a.perm_c[gj];
            // values on the last intervals [t_last, inf) of both PCFs (they
            // decide only unbounded walks, whose last window holds every
            // PCF's remaining elements)
            T vlf = T(0), vlg = T(0);
            if (!bounded) {
                const int wr_last = kAdapt ? split_wr(sSplit) : W;
                const int wc_last = kAdapt ? split_wc(sSplit, wr_last) : W;
                vlf = WF::val(*reinterpret_cast<const E*>(
                    smem + (kAdapt ? slot_base(pf, wr_last, wc_last) : even_base_f) +
                    (unsigned)(sLen[pf] - 1 - sS[pf]) * kRow));
                vlg = WF::val(*reinterpret_cast<const E*>(
                    smem + (kAdapt ? slot_base(pg, wr_last, wc_last) : even_base_g) +
                    (unsigned)(sLen[pg] - 1 - sS[pg]) * kRow));
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const int MI = combo_metric(COMBO, m);
                double I = acc.value(m);
                const T h = (MI == MI_GRAM) ? vlf * vlg : fabs(vlf - vlg);
                if (!bounded && h != T(0)) I = (h > T(0)) ? (double)INFINITY : -(double)INFINITY;
                const double F = finalize_root(a.metric[m], a.root[m], a.p[m], I);
                void* out = a.out[m];
                auto put = [&](int64_t idx) {
                    if (a.out_f64) reinterpret_cast<double*>(out)[idx] = F;
                    else reinterpret_cast<float*>(out)[idx] = (float)F;
                };
                if (!a.symmetric) {
                    put(i * a.ld_out + j);
                } else if (a.layout == PCF_OUT_FULL) {
                    put(i * a.ld_out + j);
                    if (bi != bj) put(j * a.ld_out + i);
                } else if (a.layout == kOutRowsInputColsSorted) {
                    put(i * a.ld_out + gj);
                    if (bi != bj) put(j * a.ld_out + gi);
                } else if (a.layout == PCF_OUT_FULL_SORTED) {
                    put(gi * a.ld_out + gj);
                    if (bi != bj) put(gj * a.ld_out + gi);
                } else {
                    const int64_t N = a.ld_out;
                    const int64_t lo2 = i < j ? i : j, hi2 = i < j ? j : i;
                    if (bi != bj || i <= j) put(lo2 * N - lo2 * (lo2 - 1) / 2 + (hi2 - lo2));
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int PREC, int THREADS, int CTAS = 1024 / THREADS, int WEIGHT = 0,
          bool KEYED = false>
cudaError_t launch_walk_tt(int combo, const WalkArgs& a, int grid, size_t smem, cudaStream_t s)
{
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, THREADS, smem, s>>>(a);
        return cudaGetLastError();
    };
    switch (combo) {
    case kComboL1: return go(walk_kernel<T, PREC, kComboL1, THREADS, CTAS, WEIGHT, KEYED>);
    case kComboL2: return go(walk_kernel<T, PREC, kComboL2, THREADS, CTAS, WEIGHT, KEYED>);
    case kComboGram: return go(walk_kernel<T, PREC, kComboGram, THREADS, CTAS, WEIGHT, KEYED>);
    case kComboLP: return go(walk_kernel<T, PREC, kComboLP, THREADS, CTAS, WEIGHT, KEYED>);
    case kComboL3: return go(walk_kernel<T, PREC, kComboL3, THREADS, CTAS, WEIGHT, KEYED>);
    case kComboL1L2Gram: return go(walk_kernel<T, PREC, kComboL1L2Gram, THREADS, CTAS, WEIGHT, KEYED>);
    case kComboL1L2L3: return go(walk_kernel<T, PREC, kComboL1L2L3, THREADS, CTAS, WEIGHT, KEYED>);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pcfgb
