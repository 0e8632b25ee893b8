// reduce.cu -- reductions of PCFs on the GPU (Sec. 4).
//
// ReducePair (Alg. 4) produces the PCF h_*(f, g): it walks the rectangles of
// f and g (Alg. 1) and appends the breakpoint (R.l, h(v_f, v_g)) of each
// rectangle R whose value differs from the previous rectangle's, or whose
// left end is 0.  A group of m PCFs is reduced by a binary tree (Fig. 2 with
// two inputs per node): on each level item k of the next level is
// ReducePair(item 2k, item 2k + 1) and an odd last item moves up unchanged.
// The mean is the sum divided by m; the sample standard deviation of
// Sec. 2.1 is sqrt( (1/(m - 1)) sum_i (f_i - mean)^2 ), every (f_i - mean)^2
// a ReducePair with h = (a - b)^2 and the sum a tree again.  All arithmetic
// is float64; a tree of the same shape in float64 gives the same bits.
//
// GPU design.  One tree level (or one batch of pairs) is a single merge-and-
// compact pass over a flat space of merge positions: output PCF p owns
// n_a(p) + n_b(p) positions, one per input breakpoint, in the order of the
// merge of its two breakpoint lists (ties: f's breakpoint first).  Position
// q keeps a breakpoint when it is the last position with its time (so every
// time of the union appears once) and either t = 0 or the value
// h(f(t), g(t)) differs from h(f(t-), g(t-)) -- exactly the rows Alg. 4
// inserts, decided locally from the two lists.  Persistent CTAs take chunks
// of 2048 consecutive positions by ticket (8 per thread); a thread finds its
// output PCF by binary search between the chunk's partition bounds and its
// place in the merge by a merge-path search along the diagonal, then walks
// its 8 positions.  The CTA's kept rows go to shared memory, their output
// position comes from a decoupled look-back over the chunks before it, and
// they are written in order.  No host synchronization between levels: grids
// are sized for the host-known bound on positions and read the actual number
// from device memory.  (Chunk shapes of 128 x 16 and 512 x 4 positions were
// slower: longer serial walks, or one CTA per SM.)
#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace pcfgb {
namespace {

constexpr int kRpThreads = 256;
constexpr int kRpItems = 8;
constexpr int kRpChunk = kRpThreads * kRpItems;

// Which two PCFs feed output p.
enum RpMode : int {
    kModeTree = 0,   // tree level: inputs 2k, 2k + 1 of each group of c_in (set A)
    kModeBcast = 1,  // A row p with B row p / m
    kModePair = 2,   // A row p with B row p
    kModeMap = 3     // A row p alone, values mapped
};

// Combination functions (PCF_OP_*) and value maps.
enum RpOp : int {
    kOpAdd = 0, kOpSub = 1, kOpMul = 2, kOpMax = 3, kOpMin = 4, kOpSqdiff = 5,
    kOpCopy = 8, kOpDiv = 9, kOpSqrtDiv = 10
};

struct RpArgs {
    const int64_t* a_off; const double2* a_el;   // set A, breakpoint form (t, v)
    const int64_t* b_off; const double2* b_el;   // set B (BCAST / PAIR)
    int mode, op;
    double s;                 // divisor of the value maps
    int64_t P;                // output PCFs
    int64_t c_in, c_out;      // TREE: items per group on this level and the next
    int64_t m;                // BCAST: A rows per B row
    int64_t* out_off;         // [P + 1]
    double2* out_el;          // AoS output, or
    double* out_t; double* out_v;   // SoA output (out_t != nullptr)
    int64_t out_cap;          // rows available in the output
    unsigned long long* state;  // [nchunk_cap + 1]: ticket, then chunk states (zeroed)
    int64_t* part;              // [nchunk_cap]: first output PCF of each chunk
    int64_t nchunk_cap;
    unsigned long long div_M;   // p / (c_out or m) = (p * div_M) >> div_s, p < 2^31
    int div_s;
    Header* hdr;
    unsigned long long* stats;  // [0] merge positions, [1] rows written (per call)
};

__device__ __forceinline__ double rp_h(int op, double a, double b)
{
    switch (op) {
    case kOpAdd: return __dadd_rn(a, b);
    case kOpSub: return __dsub_rn(a, b);
    case kOpMul: return __dmul_rn(a, b);
    case kOpMax: return a >= b ? a : b;
    case kOpMin: return a <= b ? a : b;
    default: { const double d = __dsub_rn(a, b); return __dmul_rn(d, d); }
    }
}

__device__ __forceinline__ double rp_map(int op, double v, double s)
{
    if (op == kOpDiv) return v / s;
    if (op == kOpSqrtDiv) return sqrt(v / s);
    return v;
}

// p / d for 0 <= p < 2^31 by multiply and shift: with s = 31 + ceil(log2 d)
// and M = ceil(2^s / d), p*M/2^s exceeds p/d by less than 2^31/2^s <= 1/d,
// which never reaches the next integer.
__device__ __forceinline__ int64_t rp_div(const RpArgs& a, int64_t p)
{
    return (int64_t)(((unsigned long long)p * a.div_M) >> a.div_s);
}

// First merge position of output p (p = P gives the total).
__device__ __forceinline__ int64_t rp_item_off(const RpArgs& a, int64_t p)
{
    switch (a.mode) {
    case kModeTree: {
        const int64_t g = rp_div(a, p), k = p - g * a.c_out;
        return a.a_off[g * a.c_in + 2 * k];
    }
    case kModeBcast: {
        const int64_t g = rp_div(a, p), r = p - g * a.m;
        int64_t o = a.a_off[p] + a.m * a.b_off[g];
        if (r) o += r * (a.b_off[g + 1] - a.b_off[g]);
        return o;
    }
    case kModePair: return a.a_off[p] + a.b_off[p];
    default: return a.a_off[p];
    }
}

// Breakpoint ranges of output p's operands; nb = 0 when p has one operand.
__device__ __forceinline__ void rp_operands(const RpArgs& a, int64_t p, const double2*& A,
                                            int64_t& na, const double2*& B, int64_t& nb)
{
    int64_t a0, a1, b0 = 0, b1 = 0;
    const double2* bel = a.b_el;
    switch (a.mode) {
    case kModeTree: {
        const int64_t g = rp_div(a, p), k = p - g * a.c_out;
        const int64_t ia = g * a.c_in + 2 * k;
        a0 = a.a_off[ia]; a1 = a.a_off[ia + 1];
        if (2 * k + 1 < a.c_in) { b0 = a1; b1 = a.a_off[ia + 2]; }
        bel = a.a_el;
        break;
    }
    case kModeBcast: {
        const int64_t g = rp_div(a, p);
        a0 = a.a_off[p]; a1 = a.a_off[p + 1]; b0 = a.b_off[g]; b1 = a.b_off[g + 1];
        break;
    }
    case kModePair:
        a0 = a.a_off[p]; a1 = a.a_off[p + 1]; b0 = a.b_off[p]; b1 = a.b_off[p + 1];
        break;
    default:
        a0 = a.a_off[p]; a1 = a.a_off[p + 1];
        break;
    }
    A = a.a_el + a0; na = a1 - a0;
    B = bel + b0; nb = b1 - b0;
}

// Largest p in [lo, hi] with rp_item_off(p) <= q.
__device__ __forceinline__ int64_t rp_find(const RpArgs& a, int64_t q, int64_t lo, int64_t hi)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (rp_item_off(a, mid) <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Exclusive block scan of one int per thread (kRpThreads threads); also returns the
// block total.
__device__ __forceinline__ int rp_block_scan(int x, int& total, int* warp_sums)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kRpThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kRpThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    total = warp_sums[kRpThreads / 32 - 1];
    const int before = warp ? warp_sums[warp - 1] : 0;
    return before + v - x;
}

// Times are non-negative (t_0 = -0.0 is stored as +0.0), so their float64
// bit patterns order like the values and compare on the integer pipe.
__device__ __forceinline__ long long tkey(double t) { return __double_as_longlong(t); }

// a == b as float64 values (+0 == -0, NaN != NaN), on the integer pipe.
__device__ __forceinline__ bool vsame(double a, double b)
{
    const unsigned long long x = (unsigned long long)__double_as_longlong(a);
    const unsigned long long y = (unsigned long long)__double_as_longlong(b);
    const bool not_nan = (x & 0x7fffffffffffffffull) <= 0x7ff0000000000000ull;
    return (x == y && not_nan) || ((x | y) << 1) == 0;
}

// Chunk states of the single-pass scan: flag in bits 62-63, value below.
constexpr unsigned long long kStAgg = 1ull << 62;    // the chunk's own row count
constexpr unsigned long long kStIncl = 2ull << 62;   // rows of chunks 0..c
constexpr unsigned long long kStErr = 3ull << 62;    // gave up: successors stop too
constexpr unsigned long long kStVal = (1ull << 62) - 1;
// Polls before a wait gives up, per group of 32 predecessors: at least
// 0.27 s in the 64 ns sleeps alone.  A predecessor holds a lower ticket, so it
// is already running and publishes within microseconds unless its SM is
// time-sliced to another process's context; such slices last milliseconds,
// two orders of magnitude below the limit.
constexpr long long kSpinPolls = 1ll << 22;

// Output position of chunk c's first row (decoupled look-back by one warp,
// every lane calls this): publish this chunk's count, then read the states
// of 32 predecessors at a time, add the counts of those up to the nearest one
// that has published its inclusive prefix, and publish ours.  Chunks are
// taken in ticket order, so every predecessor is running or done; each wait
// is bounded and an error anywhere makes the waiters give up (poison state).
// The sums are of integers, so their order does not matter.  Returns -1 on
// giving up.
__device__ long long rp_look_back(const RpArgs& a, long long c, int count,
                                  long long max_polls = kSpinPolls)
{
    const int lane = threadIdx.x & 31;
    unsigned long long* st = a.state + 1;
    if (c == 0) {
        if (lane == 0) atomicExch(&st[0], kStIncl | (unsigned long long)count);
        return 0;
    }
    if (lane == 0) atomicExch(&st[c], kStAgg | (unsigned long long)count);
    long long excl = 0;
    bool failed = false;
    for (long long base = c - 1;; base -= 32) {
        const long long pred = base - lane;
        // before chunk 0: an inclusive prefix of 0
        unsigned long long v = pred >= 0 ? __ldcg(&st[pred]) : kStIncl;
        long long polls = 0;
        while (__any_sync(0xffffffffu, (v >> 62) == 0)) {
            ++polls;
            const bool give_up = polls > max_polls ||
                                 ((polls & 1023) == 0 && __ldcg(&a.hdr->err) != kNoError);
            if (__any_sync(0xffffffffu, give_up)) {         // the same decision in every lane
                failed = true;
                break;
            }
            __nanosleep(64);
            if ((v >> 62) == 0) v = __ldcg(&st[pred]);      // (pred >= 0 here)
        }
        if (failed || __any_sync(0xffffffffu, (v >> 62) == 3)) { failed = true; break; }
        const unsigned incl = __ballot_sync(0xffffffffu, (v >> 62) == 2);
        const int stop = incl ? __ffs(incl) - 1 : 31;          // nearest inclusive prefix
        long long val = lane <= stop ? (long long)(v & kStVal) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        excl += val;
        if (incl) break;
    }
    if (failed) {
        if (lane == 0) {
            atomicExch(&st[c], kStErr);
            record_error(a.hdr, kErrWait, c);
        }
        return -1;
    }
    if (lane == 0) atomicExch(&st[c], kStIncl | (unsigned long long)(excl + count));
    return excl;
}

// One merge-and-compact pass.  Persistent CTAs take 2048-position chunks by
// ticket; each thread walks 8 positions, the CTA counts the kept rows, finds
// their output position by look-back and writes them.
__global__ void __launch_bounds__(kRpThreads) rp_kernel(const RpArgs a)
{
    __shared__ long long sChunk, sBase;
    __shared__ int warp_sums[kRpThreads / 32];
    __shared__ double2 sRow[kRpChunk];             // rows of slot tid * 8 + k
    __shared__ int sExcl[kRpThreads];
    __shared__ unsigned sKeep[kRpThreads];
    if (block_sees_error(a.hdr)) return;
    const int64_t total = rp_item_off(a, a.P);
    const int64_t nch = (total + kRpChunk - 1) / kRpChunk;
    if (nch > a.nchunk_cap) {              // the same decision in every block
        if (blockIdx.x == 0 && threadIdx.x == 0) record_error(a.hdr, kErrCapacity, total);
        return;
    }
    const double2 inf2 = make_double2(INFINITY, 0.0);

    for (;;) {
        if (threadIdx.x == 0) sChunk = (long long)atomicAdd(a.state, 1ull);
        __syncthreads();
        const long long c = sChunk;
        if (c >= nch) break;
        const int64_t cq0 = c * kRpChunk;
        const int64_t cq1 = (cq0 + kRpChunk < total ? cq0 + kRpChunk : total) - 1;
        const int64_t p_lo = a.part[c], p_hi = c + 1 < nch ? a.part[c + 1] : a.P - 1;
        const int64_t q0 = cq0 + (int64_t)threadIdx.x * kRpItems;

        unsigned keep = 0, starts = 0;
        int64_t pstart = 0;
        if (q0 <= cq1) {
            int64_t p = rp_find(a, q0, p_lo, p_hi);
            const double2* A; const double2* B;
            int64_t na, nb;
            rp_operands(a, p, A, na, B, nb);
            // merge-path split: i of A's and j of B's breakpoints precede q0
            const int64_t d = q0 - rp_item_off(a, p);
            int64_t lo = d - nb > 0 ? d - nb : 0, hi = d < na ? d : na;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (tkey(A[mid].x) <= tkey(B[d - 1 - mid].x)) lo = mid + 1; else hi = mid;
            }
            int64_t i = lo, j = d - lo;
            double2 eA = i < na ? A[i] : inf2, eB = j < nb ? B[j] : inf2;
            // values of the breakpoints consumed last on each side
            double fA = i >= 1 ? A[i - 1].y : 0.0, fB = j >= 1 ? B[j - 1].y : 0.0;
            bool have_last = false;      // value of the previous distinct time known
            double vlast = 0.0;
#pragma unroll
            for (int k = 0; k < kRpItems; ++k) {
                if (q0 + k <= cq1) {
                    if (i + j == na + nb) {             // next output PCF
                        ++p;
                        rp_operands(a, p, A, na, B, nb);
                        i = 0; j = 0;
                        eA = A[0]; eB = nb ? B[0] : inf2;
                        have_last = false;
                    }
                    if (i + j == 0) {                    // first position of output p
                        if (!starts) pstart = p;
                        starts |= 1u << k;
                    }
                    const long long ta = tkey(eA.x), tb = tkey(eB.x);
                    const bool fromA = ta <= tb;         // ties: A's breakpoint first
                    const long long t = fromA ? ta : tb;
                    if (fromA) {
                        fA = eA.y; ++i;
                        eA = i < na ? A[i] : inf2;
                    } else {
                        fB = eB.y; ++j;
                        eB = j < nb ? B[j] : inf2;
                    }
                    const long long na_t = tkey(eA.x), nb_t = tkey(eB.x);
                    const long long tn = na_t < nb_t ? na_t : nb_t;
                    bool kp = false;
                    double v = 0.0;
                    if (tn != t) {                       // last position with this time
                        if (a.mode == kModeMap) {
                            v = rp_map(a.op, fA, a.s);
                            if (t == 0 || a.op == kOpCopy) kp = true;
                            else kp = !vsame(v, have_last ? vlast : rp_map(a.op, A[i - 2].y, a.s));
                        } else if (nb == 0) {            // odd item moving up the tree
                            v = fA;
                            kp = true;
                        } else {
                            v = rp_h(a.op, fA, fB);
                            if (t == 0) {
                                kp = true;
                            } else {
                                double vp = vlast;
                                if (!have_last) {        // values just before t, from memory
                                    const double fa = tkey(A[i - 1].x) == t ? A[i - 2].y : fA;
                                    const double gb = tkey(B[j - 1].x) == t ? B[j - 2].y : fB;
                                    vp = rp_h(a.op, fa, gb);
                                }
                                kp = !vsame(v, vp);
                            }
                        }
                        vlast = v;
                        have_last = true;
                    }
                    if (kp) {
                        keep |= 1u << k;
                        sRow[threadIdx.x * kRpItems + k] = make_double2(__longlong_as_double(t), v);
                    }
                }
            }
        }
        int block_total;
        const int excl = rp_block_scan(__popc(keep), block_total, warp_sums);
        sExcl[threadIdx.x] = excl;
        sKeep[threadIdx.x] = keep;
        if (threadIdx.x < 32) {
            const long long b = rp_look_back(a, c, block_total);
            if (threadIdx.x == 0) sBase = b;
        }
        __syncthreads();
        const long long base = sBase;
        if (base < 0) break;
        // offsets of the output PCFs that start in this thread's positions
        int64_t pc = pstart;
#pragma unroll
        for (int k = 0; k < kRpItems; ++k)
            if (starts & (1u << k)) a.out_off[pc++] = base + excl + __popc(keep & ((1u << k) - 1));
        // the chunk's rows are contiguous in the output: write them in order
        for (int o = threadIdx.x; o < block_total; o += kRpThreads) {
            int lo_t = 0, hi_t = kRpThreads - 1;       // last thread with sExcl <= o
            while (lo_t < hi_t) {
                const int mid = (lo_t + hi_t + 1) >> 1;
                if (sExcl[mid] <= o) lo_t = mid; else hi_t = mid - 1;
            }
            unsigned m = sKeep[lo_t];
            for (int r = o - sExcl[lo_t]; r > 0; --r) m &= m - 1;   // drop r lowest set bits
            if (!m) continue;                                       // (cannot happen)
            const double2 row = sRow[lo_t * kRpItems + (__ffs(m) - 1)];
            const long long pos = base + o;
            if (pos < a.out_cap) {
                if (a.out_t) { a.out_t[pos] = row.x; a.out_v[pos] = row.y; }
                else a.out_el[pos] = row;
            }
        }
        if (c == nch - 1 && threadIdx.x == 0) {
            const long long rows = base + block_total;
            a.out_off[a.P] = rows;
            if (rows > a.out_cap) record_error(a.hdr, kErrCapacity, rows);
            a.stats[0] += (unsigned long long)total;
            a.stats[1] += (unsigned long long)rows;
        }
        __syncthreads();
    }
}

// Level 0: the caller's CSR arrays as (t, v) float64 pairs.
template <typename T>
__global__ void rp_pack_kernel(const T* __restrict__ t, const T* __restrict__ v, int64_t nnz,
                               double2* __restrict__ el, const Header* hdr)
{
    if (hdr->err != kNoError) return;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        el[k] = make_double2(__longlong_as_double(__double_as_longlong((double)t[k]) &
                                                  0x7fffffffffffffffll),    // -0.0 -> +0.0
                             (double)v[k]);
}

// Self-test setup: no error recorded, ticket and chunk states zero.
__global__ void init_selftest_kernel(Header* h, unsigned long long* state)
{
    h->err = kNoError;
    state[0] = state[1] = state[2] = 0;
}

__global__ void rp_init_kernel(Header* h, unsigned long long* stats, int64_t* off0)
{
    h->err = kNoError;
    h->maxlen[0] = h->maxlen[1] = 0;
    h->tiles = 0;
    stats[0] = stats[1] = 0;
    if (off0) *off0 = 0;
}

// First output PCF of every chunk of merge positions (one thread per chunk).
__global__ void rp_part_kernel(const RpArgs a)
{
    if (a.hdr->err != kNoError) return;
    const int64_t total = rp_item_off(a, a.P);
    int64_t nch = (total + kRpChunk - 1) / kRpChunk;
    if (nch > a.nchunk_cap) nch = a.nchunk_cap;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nch;
         c += (int64_t)gridDim.x * blockDim.x)
        a.part[c] = rp_find(a, c * kRpChunk, 0, a.P - 1);
}

int rp_grid()
{
    static std::once_flag once;
    static int per_sm = 1;
    std::call_once(once, [] {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, rp_kernel, kRpThreads, 0);
        per_sm = b < 1 ? 1 : b;
    });
    return per_sm * device_sm_count();
}

// One merge-and-compact pass (a zeroed ticket/state array, then the kernel).
cudaError_t run_rp(RpArgs a, int64_t item_bound, cudaStream_t s)
{
    if (a.P == 0) return cudaSuccess;
    a.nchunk_cap = (item_bound + kRpChunk - 1) / kRpChunk;
    if (a.nchunk_cap < 1) a.nchunk_cap = 1;
    // divisor of the output index: items per group (tree) or rows per B row
    const int64_t d = a.mode == kModeTree ? a.c_out : (a.mode == kModeBcast ? a.m : 1);
    int lg = 0;
    while ((1ll << lg) < d) ++lg;
    a.div_s = 31 + lg;
    a.div_M = (unsigned long long)((((unsigned __int128)1 << a.div_s) + (unsigned __int128)(d - 1)) /
                                   (unsigned __int128)d);
    cudaError_t e = cudaMemsetAsync(a.state, 0, sizeof(unsigned long long) * (size_t)(a.nchunk_cap + 1), s);
    if (e != cudaSuccess) return e;
    int64_t pgrid = (a.nchunk_cap + 255) / 256;
    if (pgrid > (int64_t)device_sm_count() * 8) pgrid = (int64_t)device_sm_count() * 8;
    rp_part_kernel<<<(int)pgrid, 256, 0, s>>>(a);
    int64_t grid = rp_grid();
    if (grid > a.nchunk_cap) grid = a.nchunk_cap;
    rp_kernel<<<(int)grid, kRpThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// Workspace carve-up shared by the size query and the calls.
struct RpLayout {
    size_t hdr, stats, lens_a, skey_a, lens_b, skey_b, el0, el0b, offA, offB, elA, elB, mean_off, mean_el,
        chunk, part, total;
};

RpLayout rp_layout(int64_t n, int64_t nnz, int64_t nb, int64_t nnzb, int64_t groups,
                   int64_t cap_items, bool with_mean, bool tree)
{
    RpLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += align_up(bytes); return at; };
    L.hdr = take(sizeof(Header));
    L.stats = take(2 * sizeof(unsigned long long));
    L.lens_a = take(sizeof(int32_t) * (size_t)n);
    L.skey_a = take(sizeof(uint32_t) * (size_t)n);
    L.lens_b = take(sizeof(int32_t) * (size_t)nb);
    L.skey_b = take(sizeof(uint32_t) * (size_t)nb);
    L.el0 = take(sizeof(double2) * (size_t)nnz);
    L.el0b = take(sizeof(double2) * (size_t)nnzb);
    L.offA = take(tree ? sizeof(int64_t) * (size_t)(n + 1) : 0);
    L.offB = take(tree ? sizeof(int64_t) * (size_t)(n + 1) : 0);
    L.elA = take(tree ? sizeof(double2) * (size_t)cap_items : 0);
    L.elB = take(tree ? sizeof(double2) * (size_t)cap_items : 0);
    L.mean_off = take(with_mean ? sizeof(int64_t) * (size_t)(groups + 1) : 0);
    L.mean_el = take(with_mean ? sizeof(double2) * (size_t)nnz : 0);
    L.chunk = take(sizeof(unsigned long long) * (size_t)((cap_items + kRpChunk - 1) / kRpChunk + 2));
    L.part = take(sizeof(int64_t) * (size_t)((cap_items + kRpChunk - 1) / kRpChunk + 2));
    L.total = o;
    return L;
}

struct RpSet { const int64_t* off; const double2* el; };

// Per-pass scratch: ticket + chunk states, chunk partition.
struct RpScratch { unsigned long long* state; int64_t* part; };

// Binary tree over `groups` groups of c items of `src`; the root of each
// group goes to `final` (AoS or SoA per its fields).  ping/pong: level
// buffers.  Returns the set holding the result when `final` is null.
cudaError_t run_tree(int op, RpSet src, int64_t groups, int64_t c, int64_t cap_items,
                     int64_t* offA, double2* elA, int64_t* offB, double2* elB,
                     const RpArgs* final, RpScratch chunk, Header* hdr,
                     unsigned long long* stats, RpSet* result, cudaStream_t s)
{
    bool ping = true;
    while (c > 1) {
        const int64_t c_out = (c + 1) / 2;
        RpArgs a{};
        a.a_off = src.off; a.a_el = src.el;
        a.mode = kModeTree; a.op = op;
        a.P = groups * c_out; a.c_in = c; a.c_out = c_out;
        a.state = chunk.state; a.part = chunk.part; a.hdr = hdr; a.stats = stats;
        if (c_out == 1 && final) {
            a.out_off = final->out_off; a.out_el = final->out_el;
            a.out_t = final->out_t; a.out_v = final->out_v; a.out_cap = final->out_cap;
        } else {
            a.out_off = ping ? offA : offB; a.out_el = ping ? elA : elB;
            a.out_cap = cap_items;
        }
        cudaError_t e = run_rp(a, cap_items, s);
        if (e != cudaSuccess) return e;
        src.off = a.out_off; src.el = a.out_el;
        ping = !ping;
        c = c_out;
    }
    if (result) *result = src;
    return cudaSuccess;
}

int64_t std_cap_bound(int64_t nnz, int64_t m)
{
    const double b = (double)nnz * (double)(m + 1);
    return b > 9.0e18 ? (int64_t)9e18 : nnz * (m + 1);
}

bool rp_csr_ok(const pcf_csr* x)
{
    if (!x) return false;
    if (x->n < 0 || x->nnz < 0 || x->n > 0x7fffffffLL) return false;
    if (x->dtype != PCF_F32 && x->dtype != PCF_F64) return false;
    if (x->n > 0 && (x->nnz < x->n || !x->offsets || !x->times || !x->values)) return false;
    return true;
}

bool rp_out_ok(const pcf_csr_out* o)
{
    return o && o->offsets && o->capacity >= 0 && (o->capacity == 0 || (o->times && o->values));
}

cudaError_t rp_validate_pack(const pcf_csr* x, Header* hdr, int32_t* lens, uint32_t* skey,
                             int slot, double2* el, cudaStream_t s)
{
    SetView sv;
    sv.n = x->n; sv.nnz = x->nnz; sv.lens = lens; sv.skey = skey; sv.slot = slot;
    cudaError_t e = launch_validate(x->offsets, x->times, x->values, x->dtype, x->n, x->nnz, kPackF64,
                                    hdr, sv, s);
    if (e != cudaSuccess) return e;
    if (x->nnz == 0) return cudaSuccess;
    int64_t grid = (x->nnz + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (grid > cap) grid = cap;
    if (x->dtype == PCF_F64)
        rp_pack_kernel<double><<<(int)grid, 256, 0, s>>>((const double*)x->times,
            (const double*)x->values, x->nnz, el, hdr);
    else
        rp_pack_kernel<float><<<(int)grid, 256, 0, s>>>((const float*)x->times,
            (const float*)x->values, x->nnz, el, hdr);
    return cudaGetLastError();
}

}  // namespace
}  // namespace pcfgb

using namespace pcfgb;

extern "C" int pcf_reduce_workspace_size(const pcf_csr* x, int64_t group_size, int reduction,
                                         int64_t std_rows, size_t* bytes)
{
    if (!rp_csr_ok(x) || !bytes || std_rows < 0) return PCF_EINVAL;
    if (reduction < PCF_RED_SUM || reduction > PCF_RED_STD) return PCF_EINVAL;
    if (group_size < 1 || (x->n % group_size)) return PCF_EINVAL;
    const int64_t groups = x->n / group_size;
    const bool sd = reduction == PCF_RED_STD;
    int64_t cap = x->nnz;
    if (sd) cap = std_rows > x->nnz ? std_rows : (std_rows ? x->nnz : std_cap_bound(x->nnz, group_size));
    *bytes = rp_layout(x->n, x->nnz, 0, 0, groups, cap, sd, true).total;
    return PCF_OK;
}

extern "C" int pcf_reduce(const pcf_csr* x, int64_t group_size, int reduction, pcf_csr_out* out,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    if (!rp_csr_ok(x) || !rp_out_ok(out)) return PCF_EINVAL;
    if (reduction < PCF_RED_SUM || reduction > PCF_RED_STD) return PCF_EINVAL;
    if (group_size < 1 || (x->n % group_size)) return PCF_EINVAL;
    if (reduction == PCF_RED_STD && group_size < 2) return PCF_EINVAL;
    if (!workspace || ((uintptr_t)workspace % kAlign)) return PCF_ENOWS;
    const int64_t m = group_size, groups = x->n / m;
    const bool sd = reduction == PCF_RED_STD;
    // the largest intermediate capacity that the workspace holds
    int64_t cap = x->nnz;
    if (rp_layout(x->n, x->nnz, 0, 0, groups, cap, sd, true).total > workspace_bytes)
        return PCF_ENOWS;
    if (sd) {
        int64_t lo = cap, hi = std_cap_bound(x->nnz, m);
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo + 1) / 2;
            if (rp_layout(x->n, x->nnz, 0, 0, groups, mid, true, true).total <= workspace_bytes)
                lo = mid;
            else
                hi = mid - 1;
        }
        cap = lo;
    }
    const RpLayout L = rp_layout(x->n, x->nnz, 0, 0, groups, cap, sd, true);
    char* w = (char*)workspace;
    Header* hdr = (Header*)(w + L.hdr);
    int64_t* offA = (int64_t*)(w + L.offA); int64_t* offB = (int64_t*)(w + L.offB);
    double2* elA = (double2*)(w + L.elA); double2* elB = (double2*)(w + L.elB);
    double2* el0 = (double2*)(w + L.el0);
    const RpScratch chunk{(unsigned long long*)(w + L.chunk), (int64_t*)(w + L.part)};
    unsigned long long* stats = (unsigned long long*)(w + L.stats);

    rp_init_kernel<<<1, 1, 0, stream>>>(hdr, stats, out->offsets);
    if (x->n == 0) return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
    if (rp_validate_pack(x, hdr, (int32_t*)(w + L.lens_a), (uint32_t*)(w + L.skey_a), 0, el0,
                         stream) != cudaSuccess)
        return PCF_ECUDA;

    RpArgs fin{};
    fin.out_off = out->offsets; fin.out_t = out->times; fin.out_v = out->values;
    fin.out_cap = out->capacity;
    const RpSet in{x->offsets, el0};
    cudaError_t e = cudaSuccess;

    auto map_to = [&](RpSet src, int64_t P, int op, double sdiv, const RpArgs& dst,
                      int64_t bound) {
        RpArgs a{};
        a.a_off = src.off; a.a_el = src.el; a.mode = kModeMap; a.op = op; a.s = sdiv; a.P = P;
        a.out_off = dst.out_off; a.out_el = dst.out_el; a.out_t = dst.out_t; a.out_v = dst.out_v;
        a.out_cap = dst.out_cap; a.state = chunk.state; a.part = chunk.part; a.hdr = hdr; a.stats = stats;
        return run_rp(a, bound, stream);
    };

    if (reduction == PCF_RED_SUM || reduction == PCF_RED_MAX || reduction == PCF_RED_MIN) {
        const int op = reduction == PCF_RED_MAX ? kOpMax : reduction == PCF_RED_MIN ? kOpMin : kOpAdd;
        if (m == 1) e = map_to(in, groups, kOpCopy, 1.0, fin, x->nnz);
        else e = run_tree(op, in, groups, m, cap, offA, elA, offB, elB, &fin, chunk, hdr, stats,
                          nullptr, stream);
    } else {
        // the sum tree, then the values divided by m
        RpSet sum;
        e = run_tree(kOpAdd, in, groups, m, cap, offA, elA, offB, elB, nullptr, chunk, hdr, stats,
                     &sum, stream);
        if (e == cudaSuccess && reduction == PCF_RED_MEAN) {
            e = map_to(sum, groups, kOpDiv, (double)m, fin, x->nnz);
        } else if (e == cudaSuccess) {
            RpArgs mean{};
            mean.out_off = (int64_t*)(w + L.mean_off); mean.out_el = (double2*)(w + L.mean_el);
            mean.out_cap = x->nnz;
            e = map_to(sum, groups, kOpDiv, (double)m, mean, x->nnz);
            // (f_i - mean)^2 for every member, then their sum tree
            if (e == cudaSuccess) {
                RpArgs a{};
                a.a_off = x->offsets; a.a_el = el0;
                a.b_off = mean.out_off; a.b_el = mean.out_el;
                a.mode = kModeBcast; a.op = kOpSqdiff; a.m = m; a.P = x->n;
                a.out_off = offA; a.out_el = elA; a.out_cap = cap; a.state = chunk.state; a.part = chunk.part; a.hdr = hdr;
                a.stats = stats;
                e = run_rp(a, cap, stream);
            }
            RpSet ss;
            if (e == cudaSuccess)
                e = run_tree(kOpAdd, RpSet{offA, elA}, groups, m, cap, offB, elB, offA, elA,
                             nullptr, chunk, hdr, stats, &ss, stream);
            if (e == cudaSuccess) e = map_to(ss, groups, kOpSqrtDiv, (double)(m - 1), fin, cap);
        }
    }
    return e == cudaSuccess ? PCF_OK : PCF_ECUDA;
}

extern "C" int pcf_combine_workspace_size(const pcf_csr* a, const pcf_csr* b, size_t* bytes)
{
    if (!rp_csr_ok(a) || !rp_csr_ok(b) || !bytes) return PCF_EINVAL;
    if (!(b->n == a->n || b->n == 1)) return PCF_EINVAL;
    const int64_t items = b->n == a->n ? a->nnz + b->nnz : a->nnz + a->n * b->nnz;
    *bytes = rp_layout(a->n, a->nnz, b->n, b->nnz, 0, items, false, false).total;
    return PCF_OK;
}

extern "C" int pcf_combine(const pcf_csr* a, const pcf_csr* b, int op, pcf_csr_out* out,
                           void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    if (!rp_csr_ok(a) || !rp_csr_ok(b) || !rp_out_ok(out)) return PCF_EINVAL;
    if (!(b->n == a->n || b->n == 1)) return PCF_EINVAL;
    if (op < PCF_OP_ADD || op > PCF_OP_SQDIFF) return PCF_EINVAL;
    if (!workspace || ((uintptr_t)workspace % kAlign)) return PCF_ENOWS;
    const bool pair = b->n == a->n;
    const int64_t items = pair ? a->nnz + b->nnz : a->nnz + a->n * b->nnz;
    const RpLayout L = rp_layout(a->n, a->nnz, b->n, b->nnz, 0, items, false, false);
    if (L.total > workspace_bytes) return PCF_ENOWS;
    char* w = (char*)workspace;
    Header* hdr = (Header*)(w + L.hdr);
    double2* elA = (double2*)(w + L.el0);
    double2* elB = (double2*)(w + L.el0b);
    unsigned long long* stats = (unsigned long long*)(w + L.stats);
    rp_init_kernel<<<1, 1, 0, stream>>>(hdr, stats, out->offsets);
    if (a->n == 0) return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
    if (rp_validate_pack(a, hdr, (int32_t*)(w + L.lens_a), (uint32_t*)(w + L.skey_a), 0, elA,
                         stream) != cudaSuccess)
        return PCF_ECUDA;
    if (rp_validate_pack(b, hdr, (int32_t*)(w + L.lens_b), (uint32_t*)(w + L.skey_b), 1, elB,
                         stream) != cudaSuccess)
        return PCF_ECUDA;
    RpArgs r{};
    r.a_off = a->offsets; r.a_el = elA; r.b_off = b->offsets; r.b_el = elB;
    r.mode = pair ? kModePair : kModeBcast; r.op = op; r.m = a->n; r.P = a->n;
    r.out_off = out->offsets; r.out_t = out->times; r.out_v = out->values;
    r.out_cap = out->capacity; r.state = (unsigned long long*)(w + L.chunk); r.part = (int64_t*)(w + L.part); r.hdr = hdr; r.stats = stats;
    return run_rp(r, items, stream) == cudaSuccess ? PCF_OK : PCF_ECUDA;
}

extern "C" int pcf_reduce_counters(const void* workspace, cudaStream_t stream,
                                   int64_t* positions, int64_t* rows)
{
    if (!workspace || ((uintptr_t)workspace % kAlign)) return PCF_ENOWS;
    unsigned long long st[2] = {0, 0};
    const char* w = (const char*)workspace;
    if (cudaMemcpyAsync(st, w + align_up(sizeof(Header)), sizeof st, cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess)
        return PCF_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return PCF_ECUDA;
    if (positions) *positions = (int64_t)st[0];
    if (rows) *rows = (int64_t)st[1];
    return PCF_OK;
}

namespace pcfgb {
namespace {

// Self-test of the bounded wait: chunk 1 looks back at chunk 0, which never
// publishes (its state stays 0), so the wait must give up after `polls`
// polls, record the wait error and publish the poison state.
__global__ void rp_wait_selftest_kernel(RpArgs a, long long polls)
{
    rp_look_back(a, 1, 1, polls);                     // one warp
}

}  // namespace
}  // namespace pcfgb

extern "C" int pcf_selftest_wait_timeout(int64_t polls, void* workspace, size_t workspace_bytes,
                                         cudaStream_t stream)
{
    if (polls < 1 || polls > (1ll << 20)) return PCF_EINVAL;
    const size_t need = align_up(sizeof(Header)) + align_up(3 * sizeof(unsigned long long));
    if (!workspace || ((uintptr_t)workspace % kAlign) || workspace_bytes < need) return PCF_ENOWS;
    char* w = (char*)workspace;
    Header* hdr = (Header*)w;
    unsigned long long* state = (unsigned long long*)(w + align_up(sizeof(Header)));
    RpArgs a{};
    a.hdr = hdr;
    a.state = state;
    init_selftest_kernel<<<1, 1, 0, stream>>>(hdr, state);
    rp_wait_selftest_kernel<<<1, 32, 0, stream>>>(a, (long long)polls);
    return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
}
