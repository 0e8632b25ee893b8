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
// inserts, decided locally from the two lists.  Each CTA takes chunks of
// 2048 consecutive positions (8 per thread); a thread finds its output PCF by
// binary search and its place in the merge by a merge-path search along the
// diagonal, then walks its 8 positions.  A count pass, a one-CTA exclusive
// scan over the chunk counts and a write pass (which redoes the walk and
// writes the kept rows at their global positions) give the compacted output
// and its offsets with no host synchronization between levels: grids are
// sized for the host-known upper bound on positions and read the actual
// number from device memory.
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
    int64_t* chunk;           // [nchunk_cap]: counts, then exclusive bases
    int64_t nchunk_cap;
    Header* hdr;
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

// First merge position of output p (p = P gives the total).
__device__ __forceinline__ int64_t rp_item_off(const RpArgs& a, int64_t p)
{
    switch (a.mode) {
    case kModeTree: {
        const int64_t g = p / a.c_out, k = p - g * a.c_out;
        return a.a_off[g * a.c_in + 2 * k];
    }
    case kModeBcast: {
        const int64_t g = p / a.m, r = p - g * a.m;
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
        const int64_t g = p / a.c_out, k = p - g * a.c_out;
        const int64_t ia = g * a.c_in + 2 * k;
        a0 = a.a_off[ia]; a1 = a.a_off[ia + 1];
        if (2 * k + 1 < a.c_in) { b0 = a1; b1 = a.a_off[ia + 2]; }
        bel = a.a_el;
        break;
    }
    case kModeBcast: {
        const int64_t g = p / a.m;
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

// Inclusive block scan of one int per thread (256 threads); returns the
// thread's exclusive prefix and the block total.
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
    __syncthreads();
    return before + v - x;
}

// Count pass (WRITE = false) and write pass (WRITE = true) over the chunks.
template <bool WRITE>
__global__ void __launch_bounds__(kRpThreads) rp_kernel(const RpArgs a)
{
    __shared__ int64_t sP[2];
    __shared__ int warp_sums[kRpThreads / 32];
    if (block_sees_error(a.hdr)) return;
    const int64_t total = rp_item_off(a, a.P);
    const int64_t nch = (total + kRpChunk - 1) / kRpChunk;
    if (!WRITE && blockIdx.x == 0 && threadIdx.x == 0 && nch > a.nchunk_cap)
        record_error(a.hdr, kErrCapacity, total);
    const int64_t nrun = nch < a.nchunk_cap ? nch : a.nchunk_cap;

    for (int64_t c = blockIdx.x; c < nrun; c += gridDim.x) {
        const int64_t cq0 = c * kRpChunk;
        const int64_t cq1 = (cq0 + kRpChunk < total ? cq0 + kRpChunk : total) - 1;
        if (threadIdx.x == 0) {
            const int64_t p0 = rp_find(a, cq0, 0, a.P - 1);
            sP[0] = p0;
            sP[1] = rp_find(a, cq1, p0, a.P - 1);
        }
        __syncthreads();
        const int64_t q0 = cq0 + (int64_t)threadIdx.x * kRpItems;

        unsigned keep = 0, starts = 0;
        int64_t pstart = 0;
        double kt[kRpItems], kv[kRpItems];
        if (q0 <= cq1) {
            int64_t p = rp_find(a, q0, sP[0], sP[1]);
            int64_t base = rp_item_off(a, p);
            const double2* A; const double2* B;
            int64_t na, nb;
            rp_operands(a, p, A, na, B, nb);
            // merge-path split: i of A's and j of B's breakpoints precede q0
            const int64_t d = q0 - base;
            int64_t lo = d - nb > 0 ? d - nb : 0, hi = d < na ? d : na;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (A[mid].x <= B[d - 1 - mid].x) lo = mid + 1; else hi = mid;
            }
            int64_t i = lo, j = d - lo;
            const double2 inf2 = make_double2(INFINITY, 0.0);
            double2 eA = i < na ? A[i] : inf2, eB = j < nb ? B[j] : inf2;
            double2 pA1 = i >= 1 ? A[i - 1] : inf2, pA2 = i >= 2 ? A[i - 2] : inf2;
            double2 pB1 = j >= 1 ? B[j - 1] : inf2, pB2 = j >= 2 ? B[j - 2] : inf2;
#pragma unroll
            for (int k = 0; k < kRpItems; ++k) {
                const int64_t q = q0 + k;
                if (q <= cq1) {
                    if (i + j == na + nb) {             // next output PCF
                        ++p;
                        base = rp_item_off(a, p);
                        rp_operands(a, p, A, na, B, nb);
                        i = 0; j = 0;
                        eA = A[0]; eB = nb ? B[0] : inf2;
                        pA1 = pA2 = pB1 = pB2 = inf2;
                    }
                    if (i + j == 0) {                    // first position of output p
                        if (!starts) pstart = p;
                        starts |= 1u << k;
                    }
                    const bool takeA = (j >= nb) || (i < na && eA.x <= eB.x);
                    double t;
                    if (takeA) {
                        t = eA.x;
                        pA2 = pA1; pA1 = eA; ++i;
                        eA = i < na ? A[i] : inf2;
                    } else {
                        t = eB.x;
                        pB2 = pB1; pB1 = eB; ++j;
                        eB = j < nb ? B[j] : inf2;
                    }
                    const double tn = eA.x < eB.x ? eA.x : eB.x;
                    bool kp = false;
                    double v = 0.0;
                    if (tn != t) {                       // last position with this time
                        if (a.mode == kModeMap) {
                            v = rp_map(a.op, pA1.y, a.s);
                            kp = (t == 0.0) || a.op == kOpCopy || v != rp_map(a.op, pA2.y, a.s);
                        } else if (nb == 0) {            // odd item moving up the tree
                            v = pA1.y;
                            kp = true;
                        } else {
                            v = rp_h(a.op, pA1.y, pB1.y);
                            if (t == 0.0) {
                                kp = true;
                            } else {
                                const double fa = pA1.x == t ? pA2.y : pA1.y;
                                const double gb = pB1.x == t ? pB2.y : pB1.y;
                                kp = v != rp_h(a.op, fa, gb);
                            }
                        }
                    }
                    if (kp) keep |= 1u << k;
                    kt[k] = t;
                    kv[k] = v;
                }
            }
        }
        int block_total;
        const int mine = __popc(keep);
        const int excl = rp_block_scan(mine, block_total, warp_sums);
        if (!WRITE) {
            if (threadIdx.x == 0) a.chunk[c] = block_total;
        } else {
            int64_t pos = a.chunk[c] + excl;
            int64_t pc = pstart;
#pragma unroll
            for (int k = 0; k < kRpItems; ++k) {
                if (starts & (1u << k)) a.out_off[pc++] = pos;
                if (keep & (1u << k)) {
                    if (pos < a.out_cap) {
                        if (a.out_t) { a.out_t[pos] = kt[k]; a.out_v[pos] = kv[k]; }
                        else a.out_el[pos] = make_double2(kt[k], kv[k]);
                    }
                    ++pos;
                }
            }
        }
        __syncthreads();
    }
}

// Exclusive scan of the chunk counts (one CTA); out_off[P] = total rows.
__global__ void __launch_bounds__(1024) rp_scan_kernel(const RpArgs a)
{
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t carry;
    if (block_sees_error(a.hdr)) return;
    const int64_t total = rp_item_off(a, a.P);
    int64_t nch = (total + kRpChunk - 1) / kRpChunk;
    if (nch > a.nchunk_cap) nch = a.nchunk_cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nch; base += 1024) {
        const int64_t idx = base + threadIdx.x;
        const int64_t x = idx < nch ? a.chunk[idx] : 0;
        int64_t v = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) warp_sums[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const int64_t excl = carry + (warp ? warp_sums[warp - 1] : 0) + v - x;
        if (idx < nch) a.chunk[idx] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.out_off[a.P] = carry;
        if (carry > a.out_cap) record_error(a.hdr, kErrCapacity, carry);
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
        el[k] = make_double2((double)t[k], (double)v[k]);
}

__global__ void rp_init_kernel(Header* h, int64_t* off0)
{
    h->err = kNoError;
    h->maxlen[0] = h->maxlen[1] = 0;
    h->tiles = 0;
    if (off0) *off0 = 0;
}

int rp_grid()
{
    static std::once_flag once;
    static int per_sm = 1;
    std::call_once(once, [] {
        int b0 = 0, b1 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, rp_kernel<false>, kRpThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, rp_kernel<true>, kRpThreads, 0);
        per_sm = b0 < b1 ? b0 : b1;
        if (per_sm < 1) per_sm = 1;
    });
    return per_sm * device_sm_count();
}

// One merge-and-compact pass: count, scan, write.
cudaError_t run_rp(RpArgs a, int64_t item_bound, cudaStream_t s)
{
    if (a.P == 0) return cudaSuccess;
    a.nchunk_cap = (item_bound + kRpChunk - 1) / kRpChunk;
    if (a.nchunk_cap < 1) a.nchunk_cap = 1;
    int64_t grid = rp_grid();
    if (grid > a.nchunk_cap) grid = a.nchunk_cap;
    rp_kernel<false><<<(int)grid, kRpThreads, 0, s>>>(a);
    rp_scan_kernel<<<1, 1024, 0, s>>>(a);
    rp_kernel<true><<<(int)grid, kRpThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// Workspace carve-up shared by the size query and the calls.
struct RpLayout {
    size_t hdr, lens_a, skey_a, lens_b, skey_b, el0, el0b, offA, offB, elA, elB, mean_off, mean_el,
        chunk, total;
};

RpLayout rp_layout(int64_t n, int64_t nnz, int64_t nb, int64_t nnzb, int64_t groups,
                   int64_t cap_items, bool with_mean, bool tree)
{
    RpLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += align_up(bytes); return at; };
    L.hdr = take(sizeof(Header));
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
    L.chunk = take(sizeof(int64_t) * (size_t)((cap_items + kRpChunk - 1) / kRpChunk + 1));
    L.total = o;
    return L;
}

struct RpSet { const int64_t* off; const double2* el; };

// Binary tree over `groups` groups of c items of `src`; the root of each
// group goes to `final` (AoS or SoA per its fields).  ping/pong: level
// buffers.  Returns the set holding the result when `final` is null.
cudaError_t run_tree(int op, RpSet src, int64_t groups, int64_t c, int64_t cap_items,
                     int64_t* offA, double2* elA, int64_t* offB, double2* elB,
                     const RpArgs* final, int64_t* chunk, Header* hdr, RpSet* result,
                     cudaStream_t s)
{
    bool ping = true;
    while (c > 1) {
        const int64_t c_out = (c + 1) / 2;
        RpArgs a{};
        a.a_off = src.off; a.a_el = src.el;
        a.mode = kModeTree; a.op = op;
        a.P = groups * c_out; a.c_in = c; a.c_out = c_out;
        a.chunk = chunk; a.hdr = hdr;
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
    cudaError_t e = launch_validate(x->offsets, x->times, x->values, x->dtype, x->n, x->nnz, 1,
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
    int64_t* chunk = (int64_t*)(w + L.chunk);

    rp_init_kernel<<<1, 1, 0, stream>>>(hdr, out->offsets);
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
        a.out_cap = dst.out_cap; a.chunk = chunk; a.hdr = hdr;
        return run_rp(a, bound, stream);
    };

    if (reduction == PCF_RED_SUM || reduction == PCF_RED_MAX || reduction == PCF_RED_MIN) {
        const int op = reduction == PCF_RED_MAX ? kOpMax : reduction == PCF_RED_MIN ? kOpMin : kOpAdd;
        if (m == 1) e = map_to(in, groups, kOpCopy, 1.0, fin, x->nnz);
        else e = run_tree(op, in, groups, m, cap, offA, elA, offB, elB, &fin, chunk, hdr, nullptr,
                          stream);
    } else {
        // the sum tree, then the values divided by m
        RpSet sum;
        e = run_tree(kOpAdd, in, groups, m, cap, offA, elA, offB, elB, nullptr, chunk, hdr, &sum,
                     stream);
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
                a.out_off = offA; a.out_el = elA; a.out_cap = cap; a.chunk = chunk; a.hdr = hdr;
                e = run_rp(a, cap, stream);
            }
            RpSet ss;
            if (e == cudaSuccess)
                e = run_tree(kOpAdd, RpSet{offA, elA}, groups, m, cap, offB, elB, offA, elA,
                             nullptr, chunk, hdr, &ss, stream);
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
    rp_init_kernel<<<1, 1, 0, stream>>>(hdr, out->offsets);
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
    r.out_cap = out->capacity; r.chunk = (int64_t*)(w + L.chunk); r.hdr = hdr;
    return run_rp(r, items, stream) == cudaSuccess ? PCF_OK : PCF_ECUDA;
}
