// mergepath.cuh -- warp-cooperative merge walk for few, long pairs.
//
// When a call has too few 32 x 32 tiles to occupy every SM (small N, long
// PCFs), one pair at a time is split across the 32 lanes of a warp.  The walk
// of a pair is the merge of the two sorted lists of finite interval ends
// X = te_f[0..n_f-2] and Y = te_g[0..n_g-2] (f first on equal ends, the same
// order as the tile walk).  Lane l takes the advances [s_l, s_{l+1}) of that
// merge, s_l = l * (|X| + |Y|) / 32; the number of X elements among the first
// s_l merged ones is found by a binary search along the cross diagonal
// (merge path, Green, McColl and Bader 2012).  The lane then starts at
// f-interval k, g-interval s_l - k, at the time of the last advance before it,
// and walks its share exactly like the tile walk.  Partial integrals are
// combined in float64 in a fixed lane order, so results do not depend on
// scheduling; they differ from one left-to-right sum only in rounding.
//
// Loads go through the read-only data cache; each lane streams two
// contiguous ranges, one interval element (an 8- or 16-byte vector: end time
// and value, or the keyed element of float64 input walked in float32: order
// key, end time as float32 hi + lo, value) per advance.
#pragma once

#include "walk.cuh"

namespace pcfgb {

// Pair index -> (row, column) for the persistent pair queue, longest first.
__device__ __forceinline__ void decode_pair(const WalkArgs& a, int64_t t, int64_t& i, int64_t& j)
{
    if (a.symmetric) {
        const int64_t N = a.n_r;
        const double q = 2.0 * (double)N + 1.0;
        const double disc = q * q - 8.0 * (double)t;
        int64_t m = (int64_t)((q - sqrt(disc > 0.0 ? disc : 0.0)) * 0.5);
        if (m < 0) m = 0;
        while (m > 0 && m * N - m * (m - 1) / 2 > t) --m;
        while ((m + 1) * N - (m + 1) * m / 2 <= t) ++m;
        j = N - 1 - m;
        i = j - (t - (m * N - m * (m - 1) / 2));
    } else {
        const int64_t q = t / a.n_c;
        i = a.n_r - 1 - q;
        j = a.n_c - 1 - (t - q * a.n_c);
    }
}

template <typename E>
__device__ __forceinline__ E ldg_elem(const E* p) { return __ldg(p); }
template <>
__device__ __forceinline__ KElem ldg_elem<KElem>(const KElem* p)
{
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    KElem e;
    e.k = u.x;
    e.hi = __uint_as_float(u.y);
    e.lo = __uint_as_float(u.z);
    e.v = __uint_as_float(u.w);
    return e;
}

// End-time order of the two walk forms: values (float64 through the integer
// pipe) or order keys.
template <typename K> __device__ __forceinline__ bool key_after(K x, K y) { return ends_after(x, y); }
template <> __device__ __forceinline__ bool key_after<uint32_t>(uint32_t x, uint32_t y) { return x > y; }

template <typename T, int PREC, int COMBO, bool KEYED = false>
__global__ void __launch_bounds__(256, 4) mergepath_kernel(const WalkArgs a, int64_t npairs)
{
    using WF = WalkForm<T, KEYED>;
    using E = typename WF::E;
    constexpr int NM = combo_n(COMBO);
    if (gated_off(a.gate, a.gate_want64)) return;   // the other walk of an AUTO64 call
    if (a.hdr->err != kNoError) return;
    const int lane = threadIdx.x & 31;
    const T p0 = (T)a.p[0];
    const E* R = reinterpret_cast<const E*>(a.pack_r);
    const E* C = reinterpret_cast<const E*>(a.pack_c);

    for (;;) {
        int64_t t = 0;
        if (lane == 0) t = a.shard_index + (int64_t)atomicAdd(&a.hdr->tiles, 1ull) * a.shard_count;
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= npairs) break;
        int64_t gi, gj;
        decode_pair(a, t, gi, gj);
        const E* F = R + a.poff_r[gi];
        const E* G = C + a.poff_c[gj];
        const int nf = a.slen_r[gi], ng = a.slen_c[gj];
        const int64_t lx = nf - 1, ly = ng - 1, total = lx + ly;
        const int64_t s0 = total * lane / 32, s1 = total * (lane + 1) / 32;

        Acc<PREC> acc[NM];
        if (s1 > s0) {
            // merge path: k = number of X among the first s0 merged ends
            int64_t lo = s0 - ly > 0 ? s0 - ly : 0, hi = s0 < lx ? s0 : lx;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const auto x = WF::key(ldg_elem(F + mid));
                const auto y = WF::key(ldg_elem(G + (s0 - 1 - mid)));
                if (!key_after(x, y)) lo = mid + 1; else hi = mid;
            }
            int kf = (int)lo, kg = (int)(s0 - lo);
            E ef = ldg_elem(F + kf), eg = ldg_elem(G + kg);
            if constexpr (KEYED) {
                // start time: the later of the two interval ends passed so far
                float tc = 0.f, tcl = 0.f;
                uint32_t kc = 0;
                if (kf > 0) { const KElem e = ldg_elem(F + kf - 1); tc = e.hi; tcl = e.lo; kc = e.k; }
                if (kg > 0) {
                    const KElem e = ldg_elem(G + kg - 1);
                    if (e.k > kc) { tc = e.hi; tcl = e.lo; }
                }
                for (int64_t s = s0; s < s1; ++s) {
                    if (((s - s0) & 15) == 0) {
#pragma unroll
                        for (int m = 0; m < NM; ++m) acc[m].flush();
                    }
                    const bool adv_f = ef.k <= eg.k;
                    const float hn = adv_f ? ef.hi : eg.hi, ln = adv_f ? ef.lo : eg.lo;
                    const float dt = __fadd_rn(__fsub_rn(hn, tc), __fsub_rn(ln, tcl));
                    tc = hn;
                    tcl = ln;
                    accumulate<COMBO, PREC, T>(acc, ef.v, eg.v, dt, p0);
                    if (adv_f) ef = ldg_elem(F + (++kf));
                    else eg = ldg_elem(G + (++kg));
                }
            } else {
                T tc = T(0);
                if (kf > 0) tc = ldg_elem(F + kf - 1).x;
                if (kg > 0) { const T y = ldg_elem(G + kg - 1).x; tc = ends_after(y, tc) ? y : tc; }
                for (int64_t s = s0; s < s1; ++s) {
                    if (((s - s0) & 15) == 0) {
#pragma unroll
                        for (int m = 0; m < NM; ++m) acc[m].flush();
                    }
                    const bool adv_f = !ends_after(ef.x, eg.x);
                    const T tn = adv_f ? ef.x : eg.x;
                    const T dt = tn - tc;
                    tc = tn;
                    accumulate<COMBO, PREC, T>(acc, ef.y, eg.y, dt, p0);
                    if (adv_f) ef = ldg_elem(F + (++kf));
                    else eg = ldg_elem(G + (++kg));
                }
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m].flush();
        // fixed-order float64 combine of the lane partials
        double I[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            double v = (s1 > s0) ? acc[m].value() : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            I[m] = v;
        }
        if (lane == 0) {
            const T lfv = WF::val(ldg_elem(F + nf - 1)), lgv = WF::val(ldg_elem(G + ng - 1));
            const int64_t i = a.perm_r[gi], j = a.perm_c[gj];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const int MI = combo_metric(COMBO, m);
                const T h = (MI == MI_GRAM) ? lfv * lgv : fabs(lfv - lgv);
                double Iv = I[m];
                if (h != T(0)) Iv = (h > T(0)) ? (double)INFINITY : -(double)INFINITY;
                const double Fv = finalize_root(a.metric[m], a.root[m], a.p[m], Iv);
                void* out = a.out[m];
                auto put = [&](int64_t idx) {
                    if (a.out_f64) reinterpret_cast<double*>(out)[idx] = Fv;
                    else reinterpret_cast<float*>(out)[idx] = (float)Fv;
                };
                if (!a.symmetric) {
                    put(i * a.ld_out + j);
                } else if (a.layout == PCF_OUT_FULL) {
                    put(i * a.ld_out + j);
                    if (gi != gj) put(j * a.ld_out + i);
                } else if (a.layout == kOutRowsInputColsSorted) {
                    put(i * a.ld_out + gj);
                    if (gi != gj) put(j * a.ld_out + gi);
                } else if (a.layout == PCF_OUT_FULL_SORTED) {
                    put(gi * a.ld_out + gj);
                    if (gi != gj) put(gj * a.ld_out + gi);
                } else {
                    const int64_t N = a.ld_out;
                    const int64_t lo2 = i < j ? i : j, hi2 = i < j ? j : i;
                    put(lo2 * N - lo2 * (lo2 - 1) / 2 + (hi2 - lo2));
                }
            }
        }
    }
}

template <typename T, int PREC, bool KEYED = false>
cudaError_t launch_mergepath_t(int combo, const WalkArgs& a, int64_t npairs, int grid, cudaStream_t s)
{
    switch (combo) {
    case kComboL1: mergepath_kernel<T, PREC, kComboL1, KEYED><<<grid, 256, 0, s>>>(a, npairs); break;
    case kComboL2: mergepath_kernel<T, PREC, kComboL2, KEYED><<<grid, 256, 0, s>>>(a, npairs); break;
    case kComboGram: mergepath_kernel<T, PREC, kComboGram, KEYED><<<grid, 256, 0, s>>>(a, npairs); break;
    case kComboLP: mergepath_kernel<T, PREC, kComboLP, KEYED><<<grid, 256, 0, s>>>(a, npairs); break;
    case kComboL3: mergepath_kernel<T, PREC, kComboL3, KEYED><<<grid, 256, 0, s>>>(a, npairs); break;
    case kComboL1L2Gram: mergepath_kernel<T, PREC, kComboL1L2Gram, KEYED><<<grid, 256, 0, s>>>(a, npairs); break;
    case kComboL1L2L3: mergepath_kernel<T, PREC, kComboL1L2L3, KEYED><<<grid, 256, 0, s>>>(a, npairs); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pcfgb
