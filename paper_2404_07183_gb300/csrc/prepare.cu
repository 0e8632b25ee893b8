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
template <typename T>
__global__ void validate_kernel(const int64_t* __restrict__ offsets,
                                const T* __restrict__ times, const T* __restrict__ values,
                                int64_t n, int64_t nnz_total, int whole, int walk_f32,
                                int32_t* __restrict__ lens, Header* hdr, int slot)
{
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
            if (lane == 0) lens[i] = 1;
            continue;
        }
        if (lane == 0) lens[i] = (int32_t)(o1 - o0);
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
                if (fabs((double)t) > (double)FLT_MAX || fabs((double)v) > (double)FLT_MAX)
                    record_error(hdr, kErrRange32, k);
            }
        }
    }
    // warp max then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if (lane == 0 && local_max) atomicMax(&hdr->maxlen[slot], local_max);
}

// Single-CTA stable LSD radix sort of (length, index) by length, 8-bit digits,
// followed by the exclusive scan of the sorted lengths.  Stability makes the
// permutation a function of the input alone.
constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads)
sort_scan_kernel(const int32_t* __restrict__ lens, int64_t n, Header* hdr, int slot,
                 int32_t* perm, int32_t* slen, int32_t* tmpk, int32_t* tmpv,
                 int64_t* __restrict__ poff)
{
    __shared__ unsigned int hist[256];
    __shared__ unsigned int base[256];
    __shared__ unsigned short wcnt[32][256];
    __shared__ int64_t carry_s;
    __shared__ int64_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (hdr->err != kNoError) return;

    unsigned int maxlen = hdr->maxlen[slot];
    int passes = 1;
    while (passes < 4 && (maxlen >> (8 * passes)) != 0) ++passes;

    for (int i = tid; i < 32 * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;

    // ping-pong: pass 0 reads (lens, index), writes A; then alternate A <-> B.
    // Choose buffers so that the last pass writes (slen, perm).
    int32_t* bufk[2];
    int32_t* bufv[2];
    if (passes % 2 == 1) { bufk[0] = slen; bufv[0] = perm; bufk[1] = tmpk; bufv[1] = tmpv; }
    else                 { bufk[0] = tmpk; bufv[0] = tmpv; bufk[1] = slen; bufv[1] = perm; }

    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        const int32_t* inK = (pass == 0) ? lens : bufk[(pass - 1) & 1];
        const int32_t* inV = (pass == 0) ? nullptr : bufv[(pass - 1) & 1];
        int32_t* outK = bufk[pass & 1];
        int32_t* outV = bufv[pass & 1];
        if (tid < 256) hist[tid] = 0;
        __syncthreads();
        for (int64_t i = tid; i < n; i += kSortThreads)
            atomicAdd(&hist[((unsigned)inK[i] >> shift) & 255u], 1u);
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of 256 counters by one warp (8 per lane)
            unsigned int v[8], s = 0;
            for (int q = 0; q < 8; ++q) { v[q] = hist[lane * 8 + q]; s += v[q]; }
            unsigned int incl = s;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            unsigned int run = incl - s;
            for (int q = 0; q < 8; ++q) { base[lane * 8 + q] = run; run += v[q]; }
        }
        __syncthreads();
        for (int64_t c0 = 0; c0 < n; c0 += kSortThreads) {
            const int64_t i = c0 + tid;
            const bool valid = i < n;
            int32_t key = 0, val = 0;
            unsigned int d = 256u + lane;   // unique dummy digit for idle lanes
            if (valid) {
                key = inK[i];
                val = (pass == 0) ? (int32_t)i : inV[i];
                d = ((unsigned)key >> shift) & 255u;
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
                outK[pos] = key;
                outV[pos] = val;
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
                            const int64_t* __restrict__ poff, void* packed_v, const Header* hdr)
{
    using E = typename Elem<Tin, Tw>::type;
    if (hdr->err != kNoError) return;
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

size_t set_bytes(int64_t n, int64_t nnz, int elem_bytes)
{
    size_t b = 0;
    b += 5 * align_up(sizeof(int32_t) * (size_t)n);
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
    v.tmpk = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)n));
    v.tmpv = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)n));
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

cudaError_t prepare_set(const int64_t* offsets, const void* times, const void* values,
                        int in_dtype, int64_t n, int64_t nnz_total, bool whole,
                        int walk_f64, Header* hdr, SetView& sv, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int g = grid_for_warps(n);
    if (in_dtype == PCF_F64) {
        validate_kernel<double><<<g, 256, 0, s>>>(offsets, (const double*)times,
            (const double*)values, n, nnz_total, whole, !walk_f64, sv.lens, hdr, sv.slot);
    } else {
        validate_kernel<float><<<g, 256, 0, s>>>(offsets, (const float*)times,
            (const float*)values, n, nnz_total, whole, !walk_f64, sv.lens, hdr, sv.slot);
    }
    sort_scan_kernel<<<1, kSortThreads, 0, s>>>(sv.lens, n, hdr, sv.slot, sv.perm, sv.slen,
                                                 sv.tmpk, sv.tmpv, sv.poff);
    if (in_dtype == PCF_F64) {
        if (walk_f64)
            pack_kernel<double, double><<<g, 256, 0, s>>>(offsets, (const double*)times,
                (const double*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr);
        else
            pack_kernel<double, float><<<g, 256, 0, s>>>(offsets, (const double*)times,
                (const double*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr);
    } else {
        if (walk_f64)
            pack_kernel<float, double><<<g, 256, 0, s>>>(offsets, (const float*)times,
                (const float*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr);
        else
            pack_kernel<float, float><<<g, 256, 0, s>>>(offsets, (const float*)times,
                (const float*)values, n, sv.perm, sv.slen, sv.poff, sv.packed, hdr);
    }
    return cudaGetLastError();
}

}  // namespace pcfgb
