// prepare.cu -- CSR validation, length sort and packing of a PCF collection.
//
// Input contract (Sec. 2, PCF definition and matrix storage): each PCF is
// t_0 = 0 < t_1 < ... < t_{n-1} with finite values; the packed form stores
// per PCF the "interval elements" (te_k, v_k) with te_k = t_{k+1} and
// te_{n-1} = +inf, so a merge walk reads one element per advance.  PCFs are
// packed in ascending length order so that the 32 x 32 pair tiles of the walk
// hold PCFs of similar length (the per-pair work is n_f + n_g - 1 steps).
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace pcfgb {

template <typename T>
__device__ __forceinline__ bool finite_val(T x) { return isfinite(x); }

// One warp per PCF: check offsets, t_0 = 0, strict increase, finiteness;
// write lengths and the running maximum length.
// auto64 (float64 input, PCF_PREC_AUTO64): instead of rejecting a time or
// value outside float32's range, mark the set as needing the float64 walk
// (Header::need64 bit `slot`), likewise for nonzero values below FLT_MIN and
// for gaps below 2^-30 of their time.
template <typename T>
__global__ void validate_kernel(const int64_t* __restrict__ offsets,
                                const T* __restrict__ times, const T* __restrict__ values,
                                int64_t n, int64_t nnz_total, int whole, int walk_f32,
                                int32_t* __restrict__ lens, uint32_t* __restrict__ skey,
                                Header* hdr, int slot, int auto64, int skip_on_error = 0)
{
    // a collection built by an earlier kernel of the call is only checked
    // when that kernel ran (no error recorded before it)
    if (skip_on_error && hdr->err != kNoError) return;
    bool need64 = false;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned int local_max = 0;
    for (int64_t i = warp0; i < n; i += nwarps) {
        int64_t o0 = offsets[i], o1 = offsets[i + 1];
        bool bad = !(o0 >= 0 && o1 > o0 && o1 <= nnz_total && (o1 - o0) < (1ll << 31));
        if (whole && i == 0 && o0 != 0) bad = true;
        if (whole && i == n - 1 && o1 != nnz_total) bad = true;
        if (bad) {
            if (lane == 0) record_error(hdr, kErrOffsets, i);
            if (lane == 0) { lens[i] = 1; skey[i] = 0; }
            continue;
        }
        if (lane == 0) {
            lens[i] = (int32_t)(o1 - o0);
            // time scale of the PCF: its last breakpoint, as float32 bits
            // (non-negative floats order like their bit patterns)
            const float tl = (float)times[o1 - 1];
            skey[i] = (tl > 0.f && tl < INFINITY) ? __float_as_uint(tl) : 0u;
        }
        local_max = max(local_max, (unsigned int)(o1 - o0));
        for (int64_t k = o0 + lane; k < o1; k += 32) {
            T t = times[k];
            T v = values[k];
            if (!finite_val(t)) { record_error(hdr, kErrTimeNaN, k); continue; }
            if (!finite_val(v)) { record_error(hdr, kErrValueNaN, k); continue; }
            if (k == o0) {
                if (t != T(0)) record_error(hdr, kErrT0, k);
            } else {
                T tp = times[k - 1];
                if (!(t > tp)) record_error(hdr, kErrOrder, k);
            }
            if (walk_f32 && sizeof(T) == 8) {
                const double at = fabs((double)t), av = fabs((double)v);
                const bool out = at > (double)FLT_MAX || av > (double)FLT_MAX;
                if (auto64) {
                    const bool tiny = (av != 0.0 && av < (double)FLT_MIN) ||
                                      (at != 0.0 && at < (double)FLT_MIN);
                    const bool dense = k > o0 &&
                                       ((double)t - (double)times[k - 1]) < kAuto64MinRelGap * at;
                    need64 = need64 || out || tiny || dense;
                } else if (out) {
                    record_error(hdr, kErrRange32, k);
                }
            }
        }
    }
    if (__any_sync(0xffffffffu, need64) && lane == 0) atomicOr(&hdr->need64, 1u << slot);
    // warp max then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if (lane == 0 && local_max) atomicMax(&hdr->maxlen[slot], local_max);
}

// Single-CTA stable LSD radix sort with 8-bit digits by a composite key:
// high word = length bucket (the length itself up to 256, then buckets of 32),
// low word = time scale (last breakpoint time, float bits) for PCFs longer
// than 256.  Lengths group the pairs of a tile by work; among long PCFs, the
// time scale groups PCFs whose breakpoints cover similar time ranges, so the
// shared-memory windows of a tile advance all of them together.  Stability
// makes the permutation a function of the input alone.  Followed by the
// sorted lengths and their exclusive scan.
constexpr int kSortThreads = 1024;
constexpr int kScaleSortMin = 256;

__device__ __forceinline__ uint32_t length_bucket(int32_t len)
{
    return len <= kScaleSortMin ? (uint32_t)len
                                : (uint32_t)kScaleSortMin + (uint32_t)((len - kScaleSortMin) >> 5);
}

__global__ void __launch_bounds__(kSortThreads)
sort_scan_kernel(const int32_t* __restrict__ lens, const uint32_t* __restrict__ skey, int64_t n,
                 Header* hdr, int slot, int32_t* perm, int32_t* slen, uint32_t* khi0,
                 uint32_t* klo0, int32_t* kv0, uint32_t* khi1, uint32_t* klo1, int32_t* kv1,
                 int64_t* __restrict__ poff)
{
    __shared__ unsigned int hist[256];
    __shared__ unsigned int base[256];
    __shared__ unsigned short wcnt[32][256];
    __shared__ int64_t carry_s;
    __shared__ int64_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (hdr->err != kNoError) return;

    const unsigned int maxlen = hdr->maxlen[slot];
    const bool use_scale = maxlen > (unsigned)kScaleSortMin;
    const int nlo = use_scale ? 4 : 0;
    const uint32_t maxb = length_bucket((int32_t)maxlen);
    int nhi = 1;
    while (nhi < 4 && (maxb >> (8 * nhi)) != 0) ++nhi;
    const int passes = nlo + nhi;

    for (int i = tid; i < 32 * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;

    uint32_t* bhi[2] = {khi0, khi1};
    uint32_t* blo[2] = {klo0, klo1};
    int32_t* bv[2] = {kv0, kv1};

    for (int pass = 0; pass < passes; ++pass) {
        const bool lo_digit = pass < nlo;
        const int shift = 8 * (lo_digit ? pass : pass - nlo);
        const int src = (pass - 1) & 1, dst = pass & 1;
        auto load = [&](int64_t i, uint32_t& hi, uint32_t& lo, int32_t& v) {
            if (pass == 0) {
                const int32_t len = lens[i];
                hi = length_bucket(len);
                lo = (use_scale && len > kScaleSortMin) ? skey[i] : 0u;
                v = (int32_t)i;
            } else {
                hi = bhi[src][i];
                lo = blo[src][i];
                v = bv[src][i];
            }
        };
        if (tid < 256) hist[tid] = 0;
        __syncthreads();
        for (int64_t i = tid; i < n; i += kSortThreads) {
            uint32_t hi, lo;
            int32_t v;
            load(i, hi, lo, v);
            atomicAdd(&hist[((lo_digit ? lo : hi) >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of 256 counters by one warp (8 per lane)
            unsigned int c[8], sum = 0;
            for (int q = 0; q < 8; ++q) { c[q] = hist[lane * 8 + q]; sum += c[q]; }
            unsigned int incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            unsigned int run = incl - sum;
            for (int q = 0; q < 8; ++q) { base[lane * 8 + q] = run; run += c[q]; }
        }
        __syncthreads();
        for (int64_t c0 = 0; c0 < n; c0 += kSortThreads) {
            const int64_t i = c0 + tid;
            const bool valid = i < n;
            uint32_t hi = 0, lo = 0;
            int32_t v = 0;
            unsigned int d = 256u + lane;   // unique dummy digit for idle lanes
            if (valid) {
                load(i, hi, lo, v);
                d = ((lo_digit ? lo : hi) >> shift) & 255u;
            }
            unsigned int peers = __match_any_sync(0xffffffffu, d);
            unsigned int rank = __popc(peers & ((1u << lane) - 1u));
            bool leader = (__ffs(peers) - 1) == lane;
            if (valid && leader) wcnt[warp][d] = (unsigned short)__popc(peers);
            __syncthreads();
            if (valid) {
                unsigned int off = 0;
                for (int w = 0; w < warp; ++w) off += wcnt[w][d];
                unsigned int pos = base[d] + off + rank;
                bhi[dst][pos] = hi;
                blo[dst][pos] = lo;
                bv[dst][pos] = v;
            }
            __syncthreads();
            if (tid < 256) {
                unsigned int tot = 0;
                for (int w = 0; w < 32; ++w) { tot += wcnt[w][tid]; wcnt[w][tid] = 0; }
                base[tid] += tot;
            }
            __syncthreads();
        }
    }
    const int32_t* order = bv[(passes - 1) & 1];
    for (int64_t s = tid; s < n; s += kSortThreads) {
        const int32_t v = order[s];
        perm[s] = v;
        slen[s] = lens[v];
    }
    __syncthreads();

    // exclusive scan of sorted lengths -> poff[0..n]
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += kSortThreads) {
        const int64_t i = c0 + tid;
        int64_t x = (i < n) ? (int64_t)slen[i] : 0;
        int64_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t ws = warp_sums[lane];
            int64_t wi = ws;
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            warp_sums[lane] = wi - ws;  // exclusive prefix of warps
        }
        __syncthreads();
        int64_t carry = carry_s;
        if (i < n) poff[i] = carry + warp_sums[warp] + incl - x;
        __syncthreads();
        if (tid == kSortThreads - 1) carry_s = carry + warp_sums[warp] + incl;
        __syncthreads();
    }
    if (tid == 0) poff[n] = carry_s;
}

template <typename Tin, typename Tw>
struct Elem;
template <> struct Elem<float, float> { using type = float2; };
template <> struct Elem<double, float> { using type = float2; };
template <> struct Elem<float, double> { using type = double2; };
template <> struct Elem<double, double> { using type = double2; };

// One warp per sorted PCF: write its interval elements in the walk type.
template <typename Tin, typename Tw>
__global__ void pack_kernel(const int64_t* __restrict__ offsets, const Tin* __restrict__ times,
                            const Tin* __restrict__ values, int64_t n,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ slen,
                            const int64_t* __restrict__ poff, void* packed_v, const Header* hdr,
                            const unsigned int* gate, int want64)
{
    using E = typename Elem<Tin, Tw>::type;
    if (hdr->err != kNoError || gated_off(gate, want64)) return;
    E* packed = reinterpret_cast<E*>(packed_v);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp0; s < n; s += nwarps) {
        const int64_t src = perm[s];
        const int64_t o = offsets[src];
        const int64_t len = slen[s];
        const int64_t dst = poff[s];
        for (int64_t k = lane; k < len; k += 32) {
            E e;
            e.x = (k + 1 < len) ? (Tw)times[o + k + 1] : (Tw)INFINITY;
            e.y = (Tw)values[o + k];
            packed[dst + k] = e;
        }
    }
}

// Keyed pack (float64 input, float32 walk), one warp per sorted PCF: element
// k gets te_k split into float32 hi = RN(te_k) and lo = RN(te_k - hi) (the
// difference is exact in float64) and v_k rounded to float32; its order key
// is filled in by the key sort (keys.cu), which reads the float64 bits of
// every finite te_k and the element's packed position from the sort input
// written here.  The last element (te = +inf) takes the largest key.  A
// float32 collection walked against a float64 one is packed the same way
// (its times are exact in float64: lo = 0).
template <typename Tin>
__global__ void pack_keyed_kernel(const int64_t* __restrict__ offsets,
                                  const Tin* __restrict__ times, const Tin* __restrict__ values,
                                  int64_t n, const int32_t* __restrict__ perm,
                                  const int32_t* __restrict__ slen, const int64_t* __restrict__ poff,
                                  KElem* __restrict__ packed, KeyOut ko, const Header* hdr,
                                  const unsigned int* gate, int want64)
{
    if (hdr->err != kNoError || gated_off(gate, want64)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t kbase = ko.base_poff ? ko.base_poff[ko.base_n] - ko.base_n : 0;
    for (int64_t s = warp0; s < n; s += nwarps) {
        const int64_t src = perm[s];
        const int64_t o = offsets[src];
        const int64_t len = slen[s];
        const int64_t dst = poff[s];
        for (int64_t k = lane; k < len; k += 32) {
            KElem e;
            e.v = (float)values[o + k];
            if (k + 1 < len) {
                const double te = (double)times[o + k + 1];
                const float hi = __double2float_rn(te);
                e.k = 0;
                e.hi = hi;
                e.lo = __double2float_rn(te - (double)hi);
                const int64_t j = kbase + dst - s + k;
                ko.key[j] = (uint64_t)__double_as_longlong(te + 0.0);   // -0 -> +0 (not a te)
                ko.pay[j] = ko.set_bit | (uint32_t)(dst + k);
            } else {
                e.k = kKeyInf;
                e.hi = INFINITY;
                e.lo = 0.f;
            }
            packed[dst + k] = e;
        }
    }
}

size_t set_bytes(int64_t n, int64_t nnz, int elem_bytes)
{
    size_t b = 0;
    b += 10 * align_up(sizeof(int32_t) * (size_t)n);
    b += align_up(sizeof(int64_t) * (size_t)(n + 1));
    b += align_up((size_t)elem_bytes * (size_t)nnz);
    return b;
}

SetView carve_set(char*& cur, int64_t n, int64_t nnz, int elem_bytes, int slot)
{
    SetView v;
    v.n = n; v.nnz = nnz; v.elem_bytes = elem_bytes; v.slot = slot;
    auto take = [&](size_t bytes) { char* p = cur; cur += align_up(bytes); return p; };
    v.lens = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)n));
    v.perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)n));
    v.slen = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)n));
    v.skey = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)n));
    for (int k = 0; k < 2; ++k) {
        v.khi[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)n));
        v.klo[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)n));
        v.kv[k] = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)n));
    }
    v.poff = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)(n + 1)));
    v.packed = take((size_t)elem_bytes * (size_t)nnz);
    return v;
}

static int grid_for_warps(int64_t warps)
{
    int64_t blocks = (warps * 32 + 255) / 256;
    int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

cudaError_t launch_validate(const int64_t* offsets, const void* times, const void* values,
                            int in_dtype, int64_t n, int64_t nnz_total, int form,
                            Header* hdr, SetView& sv, cudaStream_t s, int whole)
{
    if (n == 0) return cudaSuccess;
    const int g = grid_for_warps(n);
    const int walk_f32 = form != kPackF64;
    if (in_dtype == PCF_F64) {
        validate_kernel<double><<<g, 256, 0, s>>>(offsets, (const double*)times,
            (const double*)values, n, nnz_total, whole, walk_f32, sv.lens, sv.skey, hdr, sv.slot, 0);
    } else {
        validate_kernel<float><<<g, 256, 0, s>>>(offsets, (const float*)times,
            (const float*)values, n, nnz_total, whole, walk_f32, sv.lens, sv.skey, hdr, sv.slot, 0);
    }
    return cudaGetLastError();
}

cudaError_t pack_set(const int64_t* offsets, const void* times, const void* values, int in_dtype,
                     int64_t n, int form, Header* hdr, SetView& sv, cudaStream_t s,
                     const KeyOut* ko, const unsigned int* gate, int want64)
{
    if (n == 0) return cudaSuccess;
    const int g = grid_for_warps(n);
    if (form == kPackKeyed) {
        if (!ko) return cudaErrorInvalidValue;
        if (in_dtype == PCF_F64)
            pack_keyed_kernel<double><<<g, 256, 0, s>>>(offsets, (const double*)times,
                (const double*)values, n, sv.perm, sv.slen, sv.poff,
                reinterpret_cast<KElem*>(sv.packed), *ko, hdr, gate, want64);
        else
            pack_keyed_kernel<float><<<g, 256, 0, s>>>(offsets, (const float*)times,
                (const float*)values, n, sv.perm, sv.slen, sv.poff,
                reinterpret_cast<KElem*>(sv.packed), *ko, hdr, gate, want64);
    } else if (in_dtype == PCF_F64) {
        if (form == kPackF64)
            pack_kernel<double, double><<<g, 256, 0, s>>>(offsets, (const double*)times,
                (const double*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr, gate, want64);
        else
            pack_kernel<double, float><<<g, 256, 0, s>>>(offsets, (const double*)times,
                (const double*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr, gate, want64);
    } else {
        if (form == kPackF64)
            pack_kernel<float, double><<<g, 256, 0, s>>>(offsets, (const float*)times,
                (const float*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr, gate, want64);
        else
            pack_kernel<float, float><<<g, 256, 0, s>>>(offsets, (const float*)times,
                (const float*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr, gate, want64);
    }
    return cudaGetLastError();
}

cudaError_t prepare_set(const int64_t* offsets, const void* times, const void* values,
                        int in_dtype, int64_t n, int64_t nnz_total, bool whole,
                        int form, Header* hdr, SetView& sv, cudaStream_t s, const KeyOut* ko,
                        bool auto64, bool built)
{
    if (n == 0) return cudaSuccess;
    const int g = grid_for_warps(n);
    const int walk_f32 = form != kPackF64;
    const int a64 = auto64 && walk_f32 ? 1 : 0;
    if (in_dtype == PCF_F64) {
        validate_kernel<double><<<g, 256, 0, s>>>(offsets, (const double*)times,
            (const double*)values, n, nnz_total, whole, walk_f32, sv.lens, sv.skey, hdr, sv.slot,
            a64, built ? 1 : 0);
    } else {
        validate_kernel<float><<<g, 256, 0, s>>>(offsets, (const float*)times,
            (const float*)values, n, nnz_total, whole, walk_f32, sv.lens, sv.skey, hdr, sv.slot,
            a64, built ? 1 : 0);
    }
    sort_scan_kernel<<<1, kSortThreads, 0, s>>>(sv.lens, sv.skey, n, hdr, sv.slot, sv.perm, sv.slen,
                                                 sv.khi[0], sv.klo[0], sv.kv[0], sv.khi[1],
                                                 sv.klo[1], sv.kv[1], sv.poff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!a64) return pack_set(offsets, times, values, in_dtype, n, form, hdr, sv, s, ko);
    // both forms, gated on the need found by the validation of every set
    e = pack_set(offsets, times, values, in_dtype, n, form, hdr, sv, s, ko, &hdr->need64, 0);
    if (e != cudaSuccess) return e;
    return pack_set(offsets, times, values, in_dtype, n, kPackF64, hdr, sv, s, nullptr,
                    &hdr->need64, 1);
}

}  // namespace pcfgb
