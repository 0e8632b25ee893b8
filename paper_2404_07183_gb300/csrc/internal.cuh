// internal.cuh -- shared declarations of the CUDA library (not installed).
//
// Data layout in HBM (all inside the caller's workspace):
//   header   : device error key, max lengths, tile counter            (256 B)
//   per set  : lens[N] int32      lengths in input order
//              perm[N] int32      input index of the s-th PCF in sort order
//                                 (by length, then by time scale for long PCFs)
//              slen[N] int32      lengths in sorted order
//              skey[N] uint32     time-scale key (last breakpoint, float bits)
//              khi/klo/kv[2][N]   radix-sort ping-pong buffers
//              poff[N+1] int64    packed offsets (exclusive scan of slen)
//              packed[nnz]        "interval elements" in sorted order:
//                                 element k of PCF s = (te_k, v_k), the value
//                                 v_k on [t_k, te_k) with te_k = t_{k+1} and
//                                 te_{n-1} = +inf; float or double pairs, or
//                                 for float64 input walked in float32, KElem
//                                 (rank of te_k, te_k as float32 hi + lo, v_k)
//   key sort : (float64 bits of te, packed position) pairs, ping-pong, and
//              the radix histograms (keyed float32 walks only)
//   backward : gv[nnz], gt[nnz] float64 gradient accumulators (packed order)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pcf.h"

namespace pcfgb {

constexpr int kTile = 32;        // PCFs per tile side (rows and columns)
constexpr int kGroup = 16;       // PCFs interleaved per shared-memory region
constexpr int kTilePcfs = 64;    // 32 row PCFs + 32 column PCFs
constexpr int kWalkThreads = 1024;  // 32 warps: one diagonal of the tile each
constexpr size_t kAlign = 256;
// Tile queue bands: the default orders take the blocks of one side in bands
// of kTileBand and, inside a band, every block of the other side in turn
// against the band's blocks.  Each PCF of the other side is then staged from
// memory once per band rather than once per block of the first side, which
// cuts the walk's re-reads of the packed input (evicted from L2 by the
// output stream) by about kTileBand.
constexpr int kTileBand = 16;

// Device-side error key, minimum wins (~0 = no error):
//   bit 62: 0 for offsets errors (PCF index), 1 for element errors (element
//   index); bits 4..61: index; bits 0..3: reason.  So a broken offsets array
//   is reported first, then the smallest offending element.
enum ErrDetail : int {
    kErrOffsets = 1, kErrT0 = 2, kErrOrder = 3, kErrTimeNaN = 4,
    kErrValueNaN = 5, kErrRange32 = 6, kErrDense32 = 7, kErrCapacity = 8, kErrWait = 9,
    kErrWeight = 10
};
constexpr unsigned long long kNoError = ~0ull;

struct Header {
    unsigned long long err;      // error key
    unsigned int maxlen[2];      // max PCF length of set 0 / set 1
    unsigned long long tiles;    // persistent-kernel tile counter
    unsigned long long nkeys;    // keyed walks: interval ends ranked by the key sort
    unsigned int bound_key[2];   // keyed walks: order keys of the bounds a, b
    unsigned int need64;         // PCF_PREC_AUTO64: bit s set when set s needs the
                                 // float64 walk (range or time resolution)
    unsigned int pad32;
    unsigned long long pad[26];
};
static_assert(sizeof(Header) == 256, "header is 256 bytes");

#ifdef __CUDACC__
__device__ __forceinline__ void record_error(Header* h, int detail, long long index)
{
    const unsigned long long cls = detail == kErrOffsets ? 0ull : 1ull;
    const unsigned long long key = (cls << 62) |
                                   (((unsigned long long)index & ((1ull << 58) - 1)) << 4) |
                                   (unsigned long long)(detail & 15);
    atomicMin(&h->err, key);
}

// Block-uniform test of the error key, for kernels with block barriers
// whose own blocks may record an error while other blocks start: one thread
// reads it and every thread of the block gets the same answer.
__device__ __forceinline__ bool block_sees_error(const Header* h)
{
    return __syncthreads_or(threadIdx.x == 0 && h->err != kNoError) != 0;
}

// Tile t of the queue (longest PCFs first) -> (row block bi, column block bj).
// Symmetric (bi <= bj, NB blocks): line m of the triangle holds NB - m tiles
// and starts at tile m NB - m (m - 1) / 2.  Order 1: line m is row block m,
// columns NB - 1 down to m.  Order 0 (default): line m is column block
// NB - 1 - m; the lines are taken in bands of kTileBand columns c1 down to
// c0, and inside a band row blocks c1 down to 0 each take the band's columns
// from c1 down (row c1 - r of the band's top triangle takes r + 1 of them).
__device__ __forceinline__ void decode_upper_tile(int64_t NB, int64_t t, int order,
                                                  int64_t& bi, int64_t& bj)
{
    auto start = [NB](int64_t m) { return m * NB - m * (m - 1) / 2; };
    const double q = 2.0 * (double)NB + 1.0;
    const double disc = q * q - 8.0 * (double)t;
    int64_t m = (int64_t)((q - sqrt(disc > 0.0 ? disc : 0.0)) * 0.5);
    if (m < 0) m = 0;
    while (m > 0 && start(m) > t) --m;
    while (start(m + 1) <= t) ++m;
    if (order) {
        bi = m;
        bj = NB - 1 - (t - start(m));
        return;
    }
    const int64_t m0 = (m / kTileBand) * kTileBand;                // the band's first line
    const int64_t Bq = NB - m0 < kTileBand ? NB - m0 : kTileBand;  // its columns
    const int64_t c1 = NB - 1 - m0, c0 = c1 - Bq + 1;
    int64_t u = t - start(m0);
    const int64_t tri = Bq * (Bq + 1) / 2;
    if (u < tri) {
        int64_t r = 0;
        while ((r + 1) * (r + 2) / 2 <= u) ++r;
        bi = c1 - r;
        bj = c1 - (u - r * (r + 1) / 2);
    } else {
        u -= tri;
        bi = c0 - 1 - u / Bq;
        bj = c1 - u % Bq;
    }
}

// Cross (nb_r x nb_c blocks): bands of kTileBand row blocks from the last
// down; inside a band, column blocks from the last down, each against the
// band's rows from the last down.
__device__ __forceinline__ void decode_cross_tile(int64_t NBr, int64_t NBc, int64_t t,
                                                  int64_t& bi, int64_t& bj)
{
    const int64_t band = t / ((int64_t)kTileBand * NBc);
    const int64_t r1 = NBr - 1 - band * kTileBand;
    const int64_t Bq = r1 + 1 < kTileBand ? r1 + 1 : kTileBand;
    const int64_t u = t - band * (int64_t)kTileBand * NBc;
    bj = NBc - 1 - u / Bq;
    bi = r1 - u % Bq;
}
#endif

// Interval element of the keyed float32 walk (float64 input): the end time
// te as an exact order key (rank among the call's interval ends, see keys.cu)
// and as float32 hi + lo (hi = te rounded to float32, lo = te - hi rounded),
// and the value on the interval.  16 bytes, one vector load.
struct __align__(16) KElem {
    uint32_t k;
    float hi;
    float lo;
    float v;
};
constexpr uint32_t kKeyInf = 0xFFFFFFFFu;   // order key of te = +inf

// How a collection is packed for the walk.
enum PackForm : int {
    kPackF64 = 0,     // double2 (te, v): the float64 walk
    kPackF32 = 1,     // float2 (te, v): float32 walks of float32 input, or of
                      // float64 input with the times rounded (opt-in)
    kPackKeyed = 2    // KElem: float32 walks of float64 input
};
inline int pack_elem_bytes(int form) { return form == kPackF32 ? 8 : 16; }

// Scratch of the key sort (keys.cu): capacity `cap` interval ends.
struct KeySort {
    int64_t cap = 0;
    int64_t tiles = 0;
    uint64_t* key[2] = {nullptr, nullptr};
    uint32_t* pay[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;   // 256 x tiles digit counts
    uint32_t* tsum = nullptr;   // tiles + 1 distinct-key counts
    uint32_t* dsum = nullptr;   // 256 digit totals
};
size_t keysort_bytes(int64_t cap);
KeySort carve_keysort(char*& cursor, int64_t cap);
// Ranks of the interval ends of one or two packed keyed collections, written
// into their KElem.k fields.  The sort input (key[0], pay[0]) is written by
// the pack; the sorted keys end in key[0], pay[0].
cudaError_t rank_keys(const KeySort& ks, KElem* pack0, const int64_t* poff0, int64_t n0,
                      KElem* pack1, const int64_t* poff1, int64_t n1, Header* hdr, cudaStream_t s);
// Order keys of the integration bounds a, b into hdr->bound_key (after
// rank_keys, while the sorted keys are still in the workspace).
cudaError_t bound_keys(const KeySort& ks, const KElem* pack0, const KElem* pack1, double a, double b,
                       Header* hdr, cudaStream_t s);

// Device pointers of one prepared (validated, sorted, packed) collection.
struct SetView {
    int64_t n = 0;          // number of PCFs
    int64_t nnz = 0;        // upper bound on breakpoints (buffer capacity)
    int32_t* lens = nullptr;
    int32_t* perm = nullptr;
    int32_t* slen = nullptr;
    uint32_t* skey = nullptr;
    uint32_t* khi[2] = {nullptr, nullptr};
    uint32_t* klo[2] = {nullptr, nullptr};
    int32_t* kv[2] = {nullptr, nullptr};
    int64_t* poff = nullptr;
    void* packed = nullptr;
    int elem_bytes = 8;     // 8 (float pairs) or 16 (double pairs, KElem)
    int slot = 0;           // which Header::maxlen entry
};

// Where the keyed pack writes its sort input: entry key_base + poff[s] - s + k
// of `key` / `pay` for the finite interval end k of sorted PCF s, with
// payload = set_bit | packed position.  key_base = base_poff[base_n] - base_n
// (the keys of a set packed before, read on the device), or 0.
struct KeyOut {
    uint64_t* key = nullptr;
    uint32_t* pay = nullptr;
    uint32_t set_bit = 0;
    const int64_t* base_poff = nullptr;   // keys of another set come first
    int64_t base_n = 0;
};

size_t set_bytes(int64_t n, int64_t nnz, int elem_bytes);
SetView carve_set(char*& cursor, int64_t n, int64_t nnz, int elem_bytes, int slot);

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Validate + sort + pack one collection given by absolute CSR offsets
// (offsets[0..n]) into arrays of total length nnz_total.  When `whole` is set
// offsets[0] must be 0 and offsets[n] must equal nnz_total.
// auto64: the float32 form `form` is packed unless the input needs float64
// (Header::need64, set by the validation), in which case the float64 form is
// packed into the same buffer instead (both kernels are enqueued; each
// returns at once when the other form is the one needed).
// built: the collection was written by an earlier kernel of the same call,
// which skips its work after an input error; so is this validation then.
cudaError_t prepare_set(const int64_t* offsets, const void* times, const void* values,
                        int in_dtype, int64_t n, int64_t nnz_total, bool whole,
                        int form, Header* hdr, SetView& sv, cudaStream_t s,
                        const KeyOut* ko = nullptr, bool auto64 = false, bool built = false);
// The pack step alone (validation and length sort already done): used by
// cross calls that reuse B's sort but must re-rank its keys.  gate: null,
// or run only when (*gate != 0) == want64.
cudaError_t pack_set(const int64_t* offsets, const void* times, const void* values, int in_dtype,
                     int64_t n, int form, Header* hdr, SetView& sv, cudaStream_t s,
                     const KeyOut* ko, const unsigned int* gate = nullptr, int want64 = 0);

// Arguments of the tile walk kernels.
struct WalkArgs {
    // rows (set R) and columns (set C), sorted + packed
    const void* pack_r; const int64_t* poff_r; const int32_t* slen_r; const int32_t* perm_r;
    const void* pack_c; const int64_t* poff_c; const int32_t* slen_c; const int32_t* perm_c;
    int64_t n_r, n_c;
    int64_t nb_r, nb_c;      // tile blocks
    int64_t ntiles;
    int symmetric;           // pairwise: upper-triangle tiles, R == C
    int tile_order;          // symmetric tile order: 0 = column blocks from the last
                             // down, 1 = row blocks from the first up (each with its
                             // longest partner first)
    int window;              // W: staged elements per PCF per window
    Header* hdr;
    // outputs
    int nout;
    void* out[PCF_MAX_INTEGRALS];
    int metric[PCF_MAX_INTEGRALS];
    int root[PCF_MAX_INTEGRALS];
    double p[PCF_MAX_INTEGRALS];
    int layout;              // pcf_layout (pairwise) ; cross always dense block
    int out_f64;
    int64_t ld_out;          // cross: leading dimension; pairwise: N
    int64_t shard_index;     // this launch owns units u with u % shard_count == shard_index
    int64_t shard_count;     // >= 1
    double lo, hi;           // integration bounds [lo, hi], 0 <= lo < hi <= inf
    double lambda;           // weight exp(-lambda t) (weighted kernels only)
    float lo_hl[2], hi_hl[2];    // keyed walks: lo and hi as float32 hi + lo
    const unsigned int* bound_keys;  // keyed walks with bounds: order keys of lo,
                                     // hi (device); null = [0, inf)
    const unsigned int* gate;    // PCF_PREC_AUTO64: the launch returns at once unless
    int gate_want64;             // (*gate != 0) == gate_want64; null = always runs
};

#ifdef __CUDACC__
// Device-side choice between the float32 and float64 walks of an AUTO64 call.
__device__ __forceinline__ bool gated_off(const unsigned int* gate, int want64)
{
    return gate && ((*gate != 0u) != (want64 != 0));
}
#endif

// Internal output layout of the FULL pairwise matrices: rows in the input
// order, columns in the sort order, entry (i, t) = F(x_i, x[perm[t]]).  A
// tile's results then fill contiguous 128-byte row segments (whole DRAM
// sectors) instead of single entries scattered by the permutation; a
// per-row pass (permute_cols_kernel) restores the input order of the columns.
constexpr int kOutRowsInputColsSorted = 100;

// Metric combination codes compiled into the walk kernels.
enum Combo : int {
    kComboL1 = 0, kComboL2 = 1, kComboGram = 2, kComboLP = 3, kComboL3 = 4,
    kComboL1L2Gram = 5, kComboL1L2L3 = 6, kComboCount = 7
};

// Launch the persistent tile walk for one precision, CTA size and metric
// combination, or the warp-per-pair merge-path walk over `npairs` pairs.
#define PCF_DECL_WALK(name)                                                                     \
    cudaError_t launch_walk_##name##_t1024(int, const WalkArgs&, int, size_t, cudaStream_t);    \
    cudaError_t launch_walk_##name##_t512(int, const WalkArgs&, int, size_t, cudaStream_t);     \
    cudaError_t launch_walk_##name##_t512x3(int, const WalkArgs&, int, size_t, cudaStream_t);   \
    cudaError_t launch_walk_##name##_t1024w(int, const WalkArgs&, int, size_t, cudaStream_t);   \
    cudaError_t launch_mergepath_##name(int, const WalkArgs&, int64_t, int, cudaStream_t);
PCF_DECL_WALK(f64)
PCF_DECL_WALK(f32c)
PCF_DECL_WALK(f32)
PCF_DECL_WALK(f32b)
PCF_DECL_WALK(f32ck)
PCF_DECL_WALK(f32k)
PCF_DECL_WALK(f32bk)
#undef PCF_DECL_WALK
size_t walk_smem_bytes(int window, int elem_bytes);

// Adjoint.
struct BackArgs {
    const double2* pack; const int64_t* poff; const int32_t* slen; const int32_t* perm;
    int64_t n, nb, ntiles;
    const void* G; const void* F; int g_f64;
    int metric; double p; int apply_root;
    double* gv; double* gt;      // packed-order accumulators
    Header* hdr;
    int64_t shard_index, shard_count;   // this call walks tiles t with t % count == index
};
cudaError_t launch_backward(const BackArgs& a, cudaStream_t s);
cudaError_t launch_scatter_grad(const SetView& sv, const int64_t* offsets, const double* gv,
                                const double* gt, void* grad_values, void* grad_times,
                                int out_f64, Header* hdr, cudaStream_t s);

// A collection moved to the weighted time s = W(t) = int_0^t w (weight.cu).
struct WeightScratch {
    double* Wt = nullptr;      // W at the weight's breakpoints
    int64_t* lens2 = nullptr;  // lengths of the moved PCFs
    int64_t* off2 = nullptr;   // their offsets (n + 1)
    double* t2 = nullptr;      // moved breakpoints (capacity nnz + n)
    double* v2 = nullptr;      // their values
    int64_t cap = 0;
};
size_t weight_scratch_bytes(int64_t n, int64_t nnz, int64_t nw);
WeightScratch carve_weight(char*& cursor, int64_t n, int64_t nnz, int64_t nw);
cudaError_t launch_weight_move(const pcf_csr* x, const pcf_csr* w, const WeightScratch& ws,
                               Header* hdr, cudaStream_t s);

cudaError_t launch_segments(const pcf_csr* x, int functional, double p, int apply_root,
                            double lo, double hi, int precision, void* out, int out_f64,
                            Header* hdr, void* scratch, cudaStream_t s);
cudaError_t launch_validate(const int64_t* offsets, const void* times, const void* values,
                            int in_dtype, int64_t n, int64_t nnz_total, int form,
                            Header* hdr, SetView& sv, cudaStream_t s, int whole = 1);

// AUTO64 thresholds: a float64 collection needs the float64 walk when a time
// or value lies outside float32's normal range (above FLT_MAX, or nonzero
// below FLT_MIN) or when a gap t_{k+1} - t_k is below 2^-30 t_{k+1} (the
// float32 hi + lo form resolves widths to about 2^-48 t).
constexpr double kAuto64MinRelGap = 9.313225746154785e-10;   // 2^-30

int device_sm_count();
int device_smem_optin();

// Columns of rows-in-input-order matrices back to the input order (api.cu).
struct PermuteMats {
    void* mat[PCF_MAX_INTEGRALS];
    int n;
};
cudaError_t launch_inverse_perm(const int32_t* perm, int64_t n, uint32_t* pos, const Header* hdr,
                                cudaStream_t s);
cudaError_t launch_permute_cols(void* const* mats, int nmats, int64_t n, int out_f64,
                                const uint32_t* pos, const Header* hdr, cudaStream_t s,
                                const int32_t* rows = nullptr, int64_t r0 = 0, int64_t r1 = -1);
// Largest N whose row fits the permutation pass's shared memory.
bool permute_cols_fits(int64_t n, int out_f64);

}  // namespace pcfgb
