// keys.cu -- exact order keys of float64 interval ends for the float32 walks.
//
// A float32 walk over float64 input must still decide every comparison of
// Alg. 1 (which interval ends first, and ties) on the float64 times.  Rounding
// the times to float32 would merge distinct breakpoints closer than one
// float32 ulp and reorder others.  Instead every finite interval end te of
// the call's collections gets a 32-bit rank: twice the number of distinct
// end times below it, plus 2, so that equal times get equal ranks and the
// order of the ranks is the order of the times; the last interval of a PCF
// (te = +inf) has rank 0xFFFFFFFF.  A query time q that is not an interval
// end (an integration bound) gets 2 * (distinct ends below q) + 1, which
// orders it exactly against every end.  The walk then compares ranks with
// one unsigned compare, and forms interval widths from a float32 hi/lo split
// of each time (packed next to the rank).
//
// The ranks come from a device-wide stable LSD radix sort of the (time bits,
// packed position) pairs: non-negative float64 values order like their bit
// patterns read as unsigned 64-bit integers.  Eight passes of 8-bit digits;
// each pass is a histogram kernel (per tile of kSortTile keys), exclusive
// scans of each digit's counts over the tiles (a CTA per digit) and of the
// digit totals, and a scatter
// kernel that ranks the tile's keys stably (warp match, per-warp digit counts)
// and writes them to their digit's next free positions.  After the last pass
// a segmented count of distinct keys gives every sorted key its rank, written
// into the rank field of the packed element the payload names.
//
// The number of keys is known on the device only (it depends on the lengths
// of the rows a call packs); the kernels read it from the header and are
// launched for the workspace's capacity.
#include "internal.cuh"

namespace pcfgb {

constexpr int kSortThreads2 = 256;
constexpr int kSortItems = 32;
constexpr int kSortTile = kSortThreads2 * kSortItems;   // keys per tile (8,192)
constexpr int kSortWarps = kSortThreads2 / 32;

int64_t key_tiles(int64_t cap) { return cap > 0 ? (cap + kSortTile - 1) / kSortTile : 1; }

size_t keysort_bytes(int64_t cap)
{
    const int64_t tiles = key_tiles(cap);
    size_t b = 0;
    b += 2 * align_up(sizeof(uint64_t) * (size_t)(cap > 0 ? cap : 1));
    b += 2 * align_up(sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
    b += align_up(sizeof(uint32_t) * 256 * (size_t)tiles);
    b += align_up(sizeof(uint32_t) * (size_t)(tiles + 1));
    b += align_up(sizeof(uint32_t) * 256);
    return b;
}

KeySort carve_keysort(char*& cur, int64_t cap)
{
    KeySort k;
    const int64_t c = cap > 0 ? cap : 1;
    k.cap = cap;
    k.tiles = key_tiles(cap);
    auto take = [&](size_t bytes) { char* p = cur; cur += align_up(bytes); return p; };
    k.key[0] = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * (size_t)c));
    k.key[1] = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * (size_t)c));
    k.pay[0] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)c));
    k.pay[1] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)c));
    k.hist = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 256 * (size_t)k.tiles));
    k.tsum = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)(k.tiles + 1)));
    k.dsum = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 256));
    return k;
}

// Number of keys of a call: sum over its collections of (breakpoints - PCFs),
// from the packed offsets poff[n] of each set.
__global__ void count_keys_kernel(Header* hdr, const int64_t* poff0, int64_t n0,
                                  const int64_t* poff1, int64_t n1)
{
    // no keys after an input error, or when an AUTO64 call walks in float64
    if (hdr->err != kNoError || hdr->need64 != 0u) { hdr->nkeys = 0; return; }
    unsigned long long m = 0;
    if (poff0) m += (unsigned long long)(poff0[n0] - n0);
    if (poff1) m += (unsigned long long)(poff1[n1] - n1);
    hdr->nkeys = m;
}

// Digit histogram of one tile of keys, written digit-major: hist[d * tiles + t].
__global__ void __launch_bounds__(kSortThreads2)
radix_hist_kernel(const uint64_t* __restrict__ key, uint32_t* __restrict__ hist, int64_t tiles,
                  int shift, const Header* hdr)
{
    __shared__ uint32_t cnt[256];
    const int tid = threadIdx.x;
    cnt[tid] = 0;
    __syncthreads();
    const int64_t m = (int64_t)hdr->nkeys;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int lane = tid & 31;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + (int64_t)r * kSortThreads2 + tid;
        // one shared-memory atomic per distinct digit of the warp (the high
        // digits of nearby times mostly agree)
        const unsigned d = i < m ? ((unsigned)(key[i] >> shift) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < 256u && (__ffs(peers) - 1) == lane) atomicAdd(&cnt[d], (unsigned)__popc(peers));
    }
    __syncthreads();
    hist[(int64_t)tid * tiles + blockIdx.x] = cnt[tid];
}

// Exclusive scan of rows in place: CTA r scans a[r * len .. (r + 1) * len)
// (256 threads, 256 counters per round with a running carry) and writes the
// row's total to totals[r] when totals is given.  For the digit histograms a
// row is one digit's counts over the tiles.
__global__ void __launch_bounds__(256) scan_rows_kernel(uint32_t* __restrict__ a, int64_t len,
                                                        uint32_t* __restrict__ totals)
{
    __shared__ uint32_t wsum[8];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* row = a + (int64_t)blockIdx.x * len;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < len; base += 256) {
        const int64_t i = base + tid;
        const uint32_t x = i < len ? row[i] : 0u;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = carry;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (i < len) row[i] = before + incl - x;
        __syncthreads();
        if (tid == 255) carry = before + incl;
        __syncthreads();
    }
    if (tid == 0 && totals) totals[blockIdx.x] = carry;
}

// Stable scatter of one tile by the digit at `shift`: the tile's keys are
// taken in rounds of 256 (key order), ranked within the round by warp match
// and per-warp digit counts, and written after the positions the digit's
// earlier keys (earlier tiles, earlier rounds) took.
__global__ void __launch_bounds__(kSortThreads2)
radix_scatter_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ pin,
                     uint64_t* __restrict__ kout, uint32_t* __restrict__ pout,
                     const uint32_t* __restrict__ offs, const uint32_t* __restrict__ dbase,
                     int64_t tiles, int shift, const Header* hdr)
{
    __shared__ uint32_t run[256];
    __shared__ uint16_t wcnt[kSortWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t m = (int64_t)hdr->nkeys;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    run[tid] = dbase[tid] + offs[(int64_t)tid * tiles + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    if (base >= m) return;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + (int64_t)r * kSortThreads2 + tid;
        const bool valid = i < m;
        uint64_t k = 0;
        uint32_t p = 0;
        unsigned d = 256u + lane;            // distinct dummy digits for idle lanes
        if (valid) {
            k = kin[i];
            p = pin[i];
            d = (unsigned)(k >> shift) & 255u;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][d] = (uint16_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = k;
            pout[pos] = p;
        }
        __syncthreads();
        {
            uint32_t tot = 0;
            for (int w = 0; w < kSortWarps; ++w) { tot += wcnt[w][tid]; wcnt[w][tid] = 0; }
            run[tid] += tot;
        }
        __syncthreads();
        if (base + (int64_t)(r + 1) * kSortThreads2 >= m) break;   // block-uniform
    }
}

// Distinct keys per tile (a key differing from its predecessor, or the first).
__global__ void __launch_bounds__(kSortThreads2)
rank_count_kernel(const uint64_t* __restrict__ key, uint32_t* __restrict__ tsum, const Header* hdr)
{
    __shared__ uint32_t wsum[kSortWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t m = (int64_t)hdr->nkeys;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    uint32_t c = 0;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + (int64_t)r * kSortThreads2 + tid;
        if (i < m) c += (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) wsum[warp] = c;
    __syncthreads();
    if (tid == 0) {
        uint32_t s = 0;
        for (int w = 0; w < kSortWarps; ++w) s += wsum[w];
        tsum[blockIdx.x] = s;
    }
}

// Rank of every sorted key: 2 * (distinct keys up to and including it),
// written into the rank field of the packed element its payload names
// (bit 31 selects the set: 0 = set0, 1 = set1).
__global__ void __launch_bounds__(kSortThreads2)
rank_write_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ pay,
                  const uint32_t* __restrict__ tsum, KElem* pack0, KElem* pack1, const Header* hdr)
{
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t m = (int64_t)hdr->nkeys;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    if (tid == 0) carry = tsum[blockIdx.x];
    __syncthreads();
    for (int r = 0; r < kSortItems; ++r) {
        if (base + (int64_t)r * kSortThreads2 >= m) break;          // block-uniform
        const int64_t i = base + (int64_t)r * kSortThreads2 + tid;
        const uint32_t f = (i < m && (i == 0 || key[i] != key[i - 1])) ? 1u : 0u;
        uint32_t incl = f;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = carry;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (i < m) {
            const uint32_t d = before + incl;     // distinct keys in [0, i]
            const uint32_t p = pay[i];
            KElem* dst = (p >> 31) ? pack1 : pack0;
            dst[p & 0x7fffffffu].k = 2u * d;
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t s = 0;
            for (int w = 0; w < kSortWarps; ++w) s += wsum[w];
            carry += s;
        }
        __syncthreads();
    }
}

// Keys of the integration bounds a and b (one thread): 2 * (distinct ends
// below q) + 1, or + 2 when q is itself an interval end; b = inf maps to the
// rank of the last intervals.  Written to hdr->bound_key[0..1].
__global__ void bound_keys_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ pay,
                                  const KElem* pack0, const KElem* pack1, double a, double b,
                                  Header* hdr)
{
    const int64_t m = (int64_t)hdr->nkeys;
    const double q2[2] = {a, b};
    for (int w = 0; w < 2; ++w) {
        const double q = q2[w];
        if (isinf(q)) { hdr->bound_key[w] = 0xFFFFFFFFu; continue; }
        const uint64_t qb = (uint64_t)__double_as_longlong(q);
        int64_t lo = 0, hi = m;                 // first sorted key >= q
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (key[mid] < qb) lo = mid + 1; else hi = mid;
        }
        uint32_t below = 0;                      // distinct keys < q
        if (lo > 0) {
            const uint32_t p = pay[lo - 1];
            below = ((p >> 31) ? pack1 : pack0)[p & 0x7fffffffu].k / 2u;
        }
        hdr->bound_key[w] = 2u * below + ((lo < m && key[lo] == qb) ? 2u : 1u);
    }
}

cudaError_t rank_keys(const KeySort& ks, KElem* pack0, const int64_t* poff0, int64_t n0,
                      KElem* pack1, const int64_t* poff1, int64_t n1, Header* hdr, cudaStream_t s)
{
    count_keys_kernel<<<1, 1, 0, s>>>(hdr, poff0, n0, poff1, n1);
    const int64_t tiles = ks.tiles;
    int src = 0;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        radix_hist_kernel<<<(unsigned)tiles, kSortThreads2, 0, s>>>(ks.key[src], ks.hist, tiles, shift, hdr);
        // each digit's counts over the tiles, then the digit totals
        scan_rows_kernel<<<256, 256, 0, s>>>(ks.hist, tiles, ks.dsum);
        scan_rows_kernel<<<1, 256, 0, s>>>(ks.dsum, 256, nullptr);
        radix_scatter_kernel<<<(unsigned)tiles, kSortThreads2, 0, s>>>(
            ks.key[src], ks.pay[src], ks.key[1 - src], ks.pay[1 - src], ks.hist, ks.dsum, tiles,
            shift, hdr);
        src = 1 - src;
    }
    rank_count_kernel<<<(unsigned)tiles, kSortThreads2, 0, s>>>(ks.key[src], ks.tsum, hdr);
    scan_rows_kernel<<<1, 256, 0, s>>>(ks.tsum, tiles, nullptr);
    rank_write_kernel<<<(unsigned)tiles, kSortThreads2, 0, s>>>(ks.key[src], ks.pay[src], ks.tsum,
                                                                pack0, pack1, hdr);
    static_assert((8 & 1) == 0, "an even number of passes leaves the sorted keys in key[0]");
    return cudaGetLastError();
}

cudaError_t bound_keys(const KeySort& ks, const KElem* pack0, const KElem* pack1, double a, double b,
                       Header* hdr, cudaStream_t s)
{
    bound_keys_kernel<<<1, 1, 0, s>>>(ks.key[0], ks.pay[0], pack0, pack1, a, b, hdr);
    return cudaGetLastError();
}

}  // namespace pcfgb
