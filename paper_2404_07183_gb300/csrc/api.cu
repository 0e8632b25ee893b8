// api.cu -- the C ABI declared in include/pcf.h.
//
// Every entry point checks its host-visible arguments, lays out the caller's
// workspace, and enqueues on the caller's stream:
//   init header -> validate + length sort + pack (per collection)
//   -> persistent tile walk (one launch per fused metric group)
// or, for the adjoint, the recomputing gradient walk and a scatter back to
// the input order.  Nothing is allocated and nothing is synchronized.
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace pcfgb {

int device_sm_count()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

int device_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

size_t walk_smem_bytes(int window, int elem_bytes)
{
    return (size_t)4 * (size_t)window * (size_t)kGroup * (size_t)elem_bytes;
}

__global__ void init_header_kernel(Header* h, int keep_set1)
{
    h->err = kNoError;
    h->maxlen[0] = 0;
    if (!keep_set1) h->maxlen[1] = 0;
    h->need64 = keep_set1 ? (h->need64 & 2u) : 0u;   // a reused set 1 keeps its need
    h->tiles = 0;
}

// The persistent walks take work units from h->tiles upward; starting the
// counter at u0 makes a launch walk units u0 .. (its tile count) x units - 1.
__global__ void reset_tiles_kernel(Header* h, unsigned long long u0) { h->tiles = u0; }

// Rows of the FULL matrices whose pairs have all been written, copied from
// the device matrices to page-locked host matrices (device-accessible
// pointers): sorted positions s0 .. s1 - 1, i.e. original rows perm[s], each
// row_bytes long.  A CTA copies one row at a time, 16 bytes per thread (4
// when rows do not start on 16-byte boundaries).  128 threads at up to 32
// registers: one warp per SM sub-partition fits beside three 512-thread walk
// CTAs (40 registers), which leave 1,024 of each sub-partition's 16,384
// registers free.  The grid covers half the SMs: stores to host memory in
// flight on an SM slow the walk CTAs beside them, so the copy keeps about
// 150 KB in flight, enough to hide it behind the walk (measured: more in
// flight slowed the walk more than it sped the copy).
struct RowCopy {
    const char* src[PCF_MAX_INTEGRALS];
    char* dst[PCF_MAX_INTEGRALS];
    int n;
};

template <typename V>
__device__ __forceinline__ void copy_row(const V* __restrict__ src, V* __restrict__ dst, int nv)
{
    for (int k = threadIdx.x; k < nv; k += blockDim.x) dst[k] = __ldcs(src + k);
}

// After a data error the permutation was never written: nothing is copied
// (pcf_check reports the error), and a row index outside [0, n) is skipped.
__global__ void __launch_bounds__(128, 16) copy_rows_kernel(RowCopy rc, const int32_t* __restrict__ perm,
                                                            int64_t n, int64_t s0, int64_t s1,
                                                            int64_t row_bytes, int vec16,
                                                            const Header* hdr)
{
    if (block_sees_error(hdr)) return;
    for (int64_t s = s0 + blockIdx.x; s < s1; s += gridDim.x) {
        const int64_t row = perm[s];
        if (row < 0 || row >= n) continue;
        const int64_t off = row * row_bytes;
#pragma unroll
        for (int m = 0; m < PCF_MAX_INTEGRALS; ++m) {   // static indices: no local copy
            if (m >= rc.n) break;
            if (vec16)
                copy_row(reinterpret_cast<const int4*>(rc.src[m] + off),
                         reinterpret_cast<int4*>(rc.dst[m] + off), (int)(row_bytes / 16));
            else
                copy_row(reinterpret_cast<const int*>(rc.src[m] + off),
                         reinterpret_cast<int*>(rc.dst[m] + off), (int)(row_bytes / 4));
        }
    }
}

// pos[perm[s]] = s: the sorted position of every input index (after a data
// error the permutation was never written and nothing is done).
__global__ void inverse_perm_kernel(const int32_t* __restrict__ perm, int64_t n,
                                    uint32_t* __restrict__ pos, const Header* hdr)
{
    if (hdr->err != kNoError) return;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = perm[s];
        if (i >= 0 && i < n) pos[i] = (uint32_t)s;
    }
}

// Rows of a matrix whose columns are in the sort order, put back into the
// input order in place: a CTA loads one row into shared memory (coalesced,
// 16-byte vectors when aligned), then writes entry c from sorted column
// pos[c].  Reads and writes one matrix size each; pos (4N bytes) stays in L2.
// The rows are r0 .. r1 - 1, or (rows != null) rows[r0 .. r1 - 1].
template <typename V>
__global__ void __launch_bounds__(512) permute_cols_kernel(PermuteMats pm, int64_t n,
                                                           const uint32_t* __restrict__ pos,
                                                           const Header* hdr,
                                                           const int32_t* __restrict__ rows,
                                                           int64_t r0, int64_t r1)
{
    extern __shared__ __align__(16) unsigned char psm[];
    V* row_s = reinterpret_cast<V*>(psm);
    if (hdr->err != kNoError) return;
    constexpr int VEC = 16 / (int)sizeof(V);
    for (int m = 0; m < pm.n; ++m) {
        V* mat = reinterpret_cast<V*>(pm.mat[m]);
        for (int64_t k = r0 + blockIdx.x; k < r1; k += gridDim.x) {
            const int64_t r = rows ? (int64_t)rows[k] : k;
            if (r < 0 || r >= n) continue;
            V* row = mat + r * n;
            const bool vec = (n % VEC) == 0 && ((uintptr_t)row % 16) == 0;
            if (vec) {
                const int4* src = reinterpret_cast<const int4*>(row);
                int4* dst = reinterpret_cast<int4*>(row_s);
                for (int64_t c = threadIdx.x; c < n / VEC; c += blockDim.x) dst[c] = __ldcs(src + c);
            } else {
                for (int64_t c = threadIdx.x; c < n; c += blockDim.x) row_s[c] = row[c];
            }
            __syncthreads();
            if (vec) {
                int4* dst = reinterpret_cast<int4*>(row);
                for (int64_t c = threadIdx.x; c < n / VEC; c += blockDim.x) {
                    union { int4 q; V v[VEC]; } u;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) u.v[e] = row_s[pos[c * VEC + e]];
                    dst[c] = u.q;
                }
            } else {
                for (int64_t c = threadIdx.x; c < n; c += blockDim.x) row[c] = row_s[pos[c]];
            }
            __syncthreads();
        }
    }
}

// Copy of completed rows for matrices whose columns are in the sort order:
// host row r gets entry c from device column pos[c] (gathered through L2;
// the device row, 4N or 8N bytes, stays there while it is read), written in
// 16-byte pieces when aligned.  Same grid and placement as copy_rows_kernel.
template <typename V>
__global__ void __launch_bounds__(128, 16) gather_rows_kernel(RowCopy rc,
                                                              const int32_t* __restrict__ perm,
                                                              const uint32_t* __restrict__ pos,
                                                              int64_t n, int64_t s0, int64_t s1,
                                                              int vec16, const Header* hdr)
{
    if (block_sees_error(hdr)) return;
    constexpr int VEC = 16 / (int)sizeof(V);
    for (int64_t s = s0 + blockIdx.x; s < s1; s += gridDim.x) {
        const int64_t row = perm[s];
        if (row < 0 || row >= n) continue;
#pragma unroll
        for (int m = 0; m < PCF_MAX_INTEGRALS; ++m) {
            if (m >= rc.n) break;
            const V* src = reinterpret_cast<const V*>(rc.src[m]) + row * n;
            V* dst = reinterpret_cast<V*>(rc.dst[m]) + row * n;
            if (vec16) {
                for (int64_t c = threadIdx.x; c < n / VEC; c += blockDim.x) {
                    union { int4 q; V v[VEC]; } u;
#pragma unroll
                    for (int e = 0; e < VEC; ++e) u.v[e] = __ldcg(src + pos[c * VEC + e]);
                    reinterpret_cast<int4*>(dst)[c] = u.q;
                }
            } else {
                for (int64_t c = threadIdx.x; c < n; c += blockDim.x) dst[c] = __ldcg(src + pos[c]);
            }
        }
    }
}

__global__ void zero_kernel(double* a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0.0;
}

bool permute_cols_fits(int64_t n, int out_f64)
{
    const long long bytes = (long long)n * (out_f64 ? 8 : 4);
    return n > 0 && bytes + 1024 <= (long long)device_smem_optin();
}

cudaError_t launch_inverse_perm(const int32_t* perm, int64_t n, uint32_t* pos, const Header* hdr,
                                cudaStream_t s)
{
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    inverse_perm_kernel<<<(int)blocks, 256, 0, s>>>(perm, n, pos, hdr);
    return cudaGetLastError();
}

cudaError_t launch_permute_cols(void* const* mats, int nmats, int64_t n, int out_f64,
                                const uint32_t* pos, const Header* hdr, cudaStream_t s,
                                const int32_t* rows, int64_t r0, int64_t r1)
{
    if (r1 < 0) r1 = n;
    if (r1 <= r0) return cudaSuccess;
    PermuteMats pm;
    memset(&pm, 0, sizeof pm);
    pm.n = nmats;
    for (int k = 0; k < nmats; ++k) pm.mat[k] = mats[k];
    const size_t smem = (size_t)n * (out_f64 ? 8 : 4);
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int per = (int)((size_t)per_sm / (smem + 1024));
    if (per < 1) per = 1;
    if (per > 4) per = 4;
    int64_t grid = (int64_t)device_sm_count() * per;
    if (grid > r1 - r0) grid = r1 - r0;
    cudaError_t e;
    if (out_f64) {
        e = cudaFuncSetAttribute(permute_cols_kernel<double>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        permute_cols_kernel<double><<<(int)grid, 512, smem, s>>>(pm, n, pos, hdr, rows, r0, r1);
    } else {
        e = cudaFuncSetAttribute(permute_cols_kernel<float>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        permute_cols_kernel<float><<<(int)grid, 512, smem, s>>>(pm, n, pos, hdr, rows, r0, r1);
    }
    return cudaGetLastError();
}

}  // namespace pcfgb

using namespace pcfgb;

namespace {

bool csr_ok(const pcf_csr* x)
{
    if (!x) return false;
    if (x->n < 0 || x->nnz < 0 || x->n > 0x7fffffffLL) return false;
    if (x->dtype != PCF_F32 && x->dtype != PCF_F64) return false;
    if (x->n > 0) {
        if (x->nnz < x->n) return false;
        if (!x->offsets || !x->times || !x->values) return false;
    }
    return true;
}

// Precision argument: a base precision, optionally with PCF_PREC_ROUND_TIMES
// (float32 walks only).  Returns false for anything else.
struct Prec {
    int base = PCF_PREC_F64;
    bool round = false;
    bool auto64 = false;     // float32 walk unless the input needs the float64 one
};

bool parse_prec(int precision, Prec* out)
{
    const int base = precision & ~(PCF_PREC_ROUND_TIMES | PCF_PREC_AUTO64);
    if (base < PCF_PREC_F64 || base > PCF_PREC_F32_BLOCK) return false;
    const bool round = (precision & PCF_PREC_ROUND_TIMES) != 0;
    const bool auto64 = (precision & PCF_PREC_AUTO64) != 0;
    if ((round || auto64) && base == PCF_PREC_F64) return false;
    out->base = base;
    out->round = round;
    out->auto64 = auto64;
    return true;
}

// Element bytes of a call's packed buffers: an AUTO64 call may pack either
// its float32 form or the float64 one into them.
int call_elem_bytes(const Prec& p, int form)
{
    return p.auto64 ? 16 : pack_elem_bytes(form);
}

// How the call's collections are packed: float64 walk; float32 walk of
// float32 input (or of float64 input with rounded times, on request); or the
// keyed float32 walk when any collection holds float64 times.
int call_form(const Prec& p, const pcf_csr* x, const pcf_csr* y)
{
    if (p.base == PCF_PREC_F64) return kPackF64;
    if (!p.round && ((x && x->dtype == PCF_F64) || (y && y->dtype == PCF_F64))) return kPackKeyed;
    return kPackF32;
}

// Interval ends the key sort may have to rank (an upper bound).
int64_t key_capacity(const pcf_csr* x, const pcf_csr* y)
{
    return (x ? x->nnz : 0) + (y ? y->nnz : 0);
}

// float32 hi + lo split of a float64 time (as the keyed pack does on the device).
void split_time(double t, float out[2])
{
    if (std::isinf(t)) { out[0] = (float)t; out[1] = 0.f; return; }
    out[0] = (float)t;
    out[1] = (float)(t - (double)out[0]);
}

// Internal metric of one request: what the walk has to accumulate.
enum ReqKind { RK_L1, RK_L2, RK_L3, RK_LP, RK_GRAM };

int req_kind(const pcf_integral& f)
{
    switch (f.metric) {
    case PCF_L1: return RK_L1;
    case PCF_L2: return RK_L2;
    case PCF_GRAM: return RK_GRAM;
    case PCF_LP:
        if (f.p == 1.0) return RK_L1;
        if (f.p == 2.0) return RK_L2;
        if (f.p == 3.0) return RK_L3;
        return RK_LP;
    default: return -1;
    }
}

struct Launch {
    int combo;
    int idx[3];   // request index per combo slot
    int n;
};

// Group requests into walks: the fused combinations first, the rest alone.
std::vector<Launch> plan(const pcf_integral* F, int nF)
{
    std::vector<Launch> out;
    std::vector<int> kinds(nF);
    std::vector<bool> used(nF, false);
    for (int i = 0; i < nF; ++i) kinds[i] = req_kind(F[i]);
    auto find = [&](int kind) {
        for (int i = 0; i < nF; ++i) if (!used[i] && kinds[i] == kind) return i;
        return -1;
    };
    for (;;) {
        int a = find(RK_L1), b = find(RK_L2), g = find(RK_GRAM), c = find(RK_L3);
        if (a >= 0 && b >= 0 && g >= 0) {
            used[a] = used[b] = used[g] = true;
            out.push_back({kComboL1L2Gram, {a, b, g}, 3});
            continue;
        }
        if (a >= 0 && b >= 0 && c >= 0) {
            used[a] = used[b] = used[c] = true;
            out.push_back({kComboL1L2L3, {a, b, c}, 3});
            continue;
        }
        break;
    }
    for (int i = 0; i < nF; ++i) {
        if (used[i]) continue;
        int combo = kinds[i] == RK_L1 ? kComboL1 : kinds[i] == RK_L2 ? kComboL2
                  : kinds[i] == RK_L3 ? kComboL3 : kinds[i] == RK_LP ? kComboLP : kComboGram;
        out.push_back({combo, {i, -1, -1}, 1});
    }
    return out;
}

int check_requests(const pcf_integral* F, int nF, bool need_out)
{
    if (!F || nF < 1 || nF > PCF_MAX_INTEGRALS) return PCF_EINVAL;
    for (int i = 0; i < nF; ++i) {
        if (req_kind(F[i]) < 0) return PCF_EINVAL;
        if (F[i].metric == PCF_LP && !(F[i].p >= 1.0 && std::isfinite(F[i].p))) return PCF_EINVAL;
        if (need_out && !F[i].out) return PCF_EINVAL;
    }
    return PCF_OK;
}

int check_schedule(const pcf_schedule* sc)
{
    if (!sc) return PCF_OK;
    if (sc->kernel < PCF_SCHED_AUTO || sc->kernel > PCF_SCHED_TILE_512X3) return PCF_EINVAL;
    if (sc->window != 0 && sc->window < 8) return PCF_EINVAL;
    if (sc->shard_count < 0 || sc->shard_index < 0) return PCF_EINVAL;
    if (sc->shard_count > 1 && sc->shard_index >= sc->shard_count) return PCF_EINVAL;
    if (sc->shard_count <= 1 && sc->shard_index != 0) return PCF_EINVAL;
    for (int k = 0; k < 4; ++k) if (sc->reserved[k] != 0) return PCF_EINVAL;
    return PCF_OK;
}

int check_window(const pcf_window* w)
{
    if (!w) return PCF_OK;
    if (!(w->a >= 0.0) || std::isinf(w->a) || !(w->b > w->a) || std::isnan(w->b)) return PCF_EINVAL;
    if (!(w->lambda >= 0.0) || std::isinf(w->lambda)) return PCF_EINVAL;
    for (int k = 0; k < 4; ++k) if (w->reserved[k] != 0) return PCF_EINVAL;
    return PCF_OK;
}

// kernel_out: the schedule kernel the call resolves to (AUTO decided here).
// unit0: first work unit (tile schedules; the launch ends at wa.ntiles).
int run_walks(WalkArgs& wa, const pcf_integral* F, int nF, int precision, int form,
              const pcf_schedule* sched, const pcf_window* win, cudaStream_t s,
              int64_t unit0 = 0, int* kernel_out = nullptr)
{
    const int elem_bytes = pack_elem_bytes(form);
    const bool keyed = form == kPackKeyed;
    const int sms = device_sm_count();
    wa.lo = win ? win->a : 0.0;
    wa.hi = win ? win->b : (double)INFINITY;
    wa.lambda = win ? win->lambda : 0.0;
    const bool windowed = wa.lo > 0.0 || !std::isinf(wa.hi) || wa.lambda > 0.0;
    const bool weighted = wa.lambda > 0.0;
    wa.shard_count = (sched && sched->shard_count > 1) ? sched->shard_count : 1;
    wa.shard_index = (sched && sched->shard_count > 1) ? sched->shard_index : 0;
    int kernel = sched ? sched->kernel : PCF_SCHED_AUTO;
    if (kernel == PCF_SCHED_AUTO)
        kernel = (wa.ntiles * 2 < sms && !windowed) ? PCF_SCHED_MERGEPATH : PCF_SCHED_TILE_1024;
    if (windowed && kernel == PCF_SCHED_MERGEPATH) return PCF_EUNSUPPORTED;
    if (weighted && kernel != PCF_SCHED_TILE_1024) return PCF_EUNSUPPORTED;
    if (kernel_out) *kernel_out = kernel;
    if (kernel == PCF_SCHED_MERGEPATH && unit0 != 0) return PCF_EINVAL;

    int64_t grid = 0;
    size_t smem = 0;
    int64_t npairs = 0;
    if (kernel == PCF_SCHED_MERGEPATH) {
        npairs = wa.symmetric ? wa.n_r * (wa.n_r + 1) / 2 : wa.n_r * wa.n_c;
        grid = (int64_t)sms * 4;
        const int64_t need = (npairs + 7) / 8;    // 8 warps per block
        if (grid > need) grid = need;
        if (grid < 1) return PCF_OK;
    } else {
        const bool half = kernel == PCF_SCHED_TILE_512X2 || kernel == PCF_SCHED_TILE_512X3;
        const int ctas = kernel == PCF_SCHED_TILE_512X3 ? 3 : (half ? 2 : 1);
        const int regions = half ? 3 : 4;   // 32 x 16 or 32 x 32 units
        int dev = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        long budget = (long)per_sm / ctas - 1024 - 2048;       // per-CTA reserve + static
        const long optin = (long)device_smem_optin() - 2048;
        if (budget > optin) budget = optin;
        int Wmax = (int)(budget / ((long)regions * kGroup * elem_bytes));
        if (Wmax > 4096) Wmax = 4096;
        int W = (sched && sched->window) ? sched->window : Wmax;
        if (W > Wmax) return PCF_EINVAL;
        if (W < 8) return PCF_ECUDA;
        wa.window = W;
        smem = (size_t)regions * (size_t)W * kGroup * (size_t)elem_bytes;
        grid = (int64_t)sms * ctas;
        const int64_t units = wa.ntiles * (half ? 2 : 1) - unit0;
        if (grid > units) grid = units;
        if (grid < 1) return PCF_OK;
    }
    for (const Launch& L : plan(F, nF)) {
        wa.nout = L.n;
        for (int k = 0; k < L.n; ++k) {
            const pcf_integral& f = F[L.idx[k]];
            wa.out[k] = f.out;
            wa.metric[k] = f.metric;
            wa.root[k] = f.apply_root ? 1 : 0;
            wa.p[k] = f.metric == PCF_LP ? f.p : (f.metric == PCF_L2 ? 2.0 : 1.0);
        }
        reset_tiles_kernel<<<1, 1, 0, s>>>(wa.hdr, (unsigned long long)unit0);
        cudaError_t e;
        const int g = (int)grid;
        // launcher of (schedule, precision, form)
#define PCF_PICK(sfx)                                                                       \
        (precision == PCF_PREC_F64 ? launch_walk_f64_##sfx                                  \
         : precision == PCF_PREC_F32_COMP ? (keyed ? launch_walk_f32ck_##sfx : launch_walk_f32c_##sfx) \
         : precision == PCF_PREC_F32_BLOCK ? (keyed ? launch_walk_f32bk_##sfx : launch_walk_f32b_##sfx) \
         : (keyed ? launch_walk_f32k_##sfx : launch_walk_f32_##sfx))
        if (kernel == PCF_SCHED_MERGEPATH) {
            auto mp = precision == PCF_PREC_F64 ? launch_mergepath_f64
                    : precision == PCF_PREC_F32_COMP ? (keyed ? launch_mergepath_f32ck : launch_mergepath_f32c)
                    : precision == PCF_PREC_F32_BLOCK ? (keyed ? launch_mergepath_f32bk : launch_mergepath_f32b)
                    : (keyed ? launch_mergepath_f32k : launch_mergepath_f32);
            e = mp(L.combo, wa, npairs, g, s);
        } else if (kernel == PCF_SCHED_TILE_512X3) {
            e = PCF_PICK(t512x3)(L.combo, wa, g, smem, s);
        } else if (kernel == PCF_SCHED_TILE_512X2) {
            e = PCF_PICK(t512)(L.combo, wa, g, smem, s);
        } else if (weighted) {
            e = PCF_PICK(t1024w)(L.combo, wa, g, smem, s);
        } else {
            e = PCF_PICK(t1024)(L.combo, wa, g, smem, s);
        }
#undef PCF_PICK
        if (e != cudaSuccess) return PCF_ECUDA;
    }
    return PCF_OK;
}

// The walks of a call: the float32 form, or for AUTO64 both the float32 and
// the float64 walks, each gated on the device-side need (one of them returns
// at once).
int run_walks_for(WalkArgs& wa, const pcf_integral* F, int nF, const Prec& pr, int form,
                  const pcf_schedule* sched, const pcf_window* win, cudaStream_t s,
                  int64_t unit0 = 0)
{
    if (!pr.auto64 || form == kPackF64) {
        wa.gate = nullptr;
        return run_walks(wa, F, nF, pr.base, form, sched, win, s, unit0);
    }
    wa.gate = &wa.hdr->need64;
    wa.gate_want64 = 0;
    int rc = run_walks(wa, F, nF, pr.base, form, sched, win, s, unit0);
    if (rc != PCF_OK) return rc;
    WalkArgs w64 = wa;
    w64.gate_want64 = 1;
    w64.bound_keys = nullptr;
    return run_walks(w64, F, nF, PCF_PREC_F64, kPackF64, sched, win, s, unit0);
}

// Bands of the symmetric tile order for streaming a matrix to the host.  The
// walk takes the tiles (bi, bj), bi <= bj, row block by row block from the
// first (shortest PCFs) up (WalkArgs::tile_order = 1); once row blocks
// 0 .. b are done, every pair of the sorted blocks 0 .. b has been written,
// so their rows are final.  Rows then complete at a nearly even rate over
// the walk (a row block's work, n_b (NB - b) + sum of the longer blocks, falls
// only near the end), whereas the walk's default order (column blocks from
// the longest down) finishes the shortest quarter of the rows in the last
// few percent of the work, leaving their copies after the walk.  Returns the
// cumulative row-block counts 0 = M_0 < M_1 < ... = NB.  The first bands
// (copies start early) and the last ones (copied after the walk ends) are a
// quarter and a half of the others.
std::vector<int64_t> plan_bands(int64_t NB, int nbands)
{
    std::vector<int64_t> cuts{0};
    int64_t left = NB;
    auto take = [&](int64_t w) {
        if (w > left) w = left;
        if (w > 0) { cuts.push_back(cuts.back() + w); left -= w; }
    };
    if (nbands <= 1) { take(NB); return cuts; }
    const int64_t B = (NB + nbands - 1) / nbands;
    const int64_t q = B / 4 > 0 ? B / 4 : 1, h = B / 2 > 0 ? B / 2 : 1;
    take(q);
    take(h);
    while (left > h + q) take(B < left - (h + q) ? B : left - (h + q));
    take(h);
    take(q);
    take(left);
    return cuts;
}

}  // namespace

extern "C" {

int pcf_workspace_size(const pcf_csr* x, const pcf_csr* y, int precision, int purpose,
                       size_t* bytes)
{
    if (!bytes || !x || x->n < 0 || x->nnz < 0 || x->n > 0x7fffffffLL) return PCF_EINVAL;
    if (y && (y->n < 0 || y->nnz < 0 || y->n > 0x7fffffffLL)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    if (purpose != PCF_WS_FORWARD && purpose != PCF_WS_BACKWARD) return PCF_EINVAL;
    const int form = purpose == PCF_WS_BACKWARD ? kPackF64 : call_form(pr, x, y);
    const int es = purpose == PCF_WS_BACKWARD ? 16 : call_elem_bytes(pr, form);
    size_t b = sizeof(Header);
    if (y) b += set_bytes(y->n, y->nnz, es);
    b += set_bytes(x->n, x->nnz, es);
    if (form == kPackKeyed) b += keysort_bytes(key_capacity(x, y));
    if (purpose == PCF_WS_BACKWARD) b += 2 * align_up(sizeof(double) * (size_t)x->nnz);
    *bytes = b;
    return PCF_OK;
}

static int pairwise_common(const pcf_csr* x, int precision, void* workspace,
                           size_t workspace_bytes, Header** hdr_out, SetView* sv_out,
                           KeySort* ks_out = nullptr, int* form_out = nullptr)
{
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    const int form = call_form(pr, x, nullptr);
    if (form == kPackKeyed && key_capacity(x, nullptr) > 0x7fffffffLL) return PCF_EUNSUPPORTED;
    size_t need = 0;
    pcf_workspace_size(x, nullptr, precision, PCF_WS_FORWARD, &need);
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || workspace_bytes < need) return PCF_ENOWS;
    char* cur = (char*)workspace;
    *hdr_out = (Header*)cur;
    cur += sizeof(Header);
    *sv_out = carve_set(cur, x->n, x->nnz, call_elem_bytes(pr, form), 0);
    if (form == kPackKeyed && ks_out) *ks_out = carve_keysort(cur, key_capacity(x, nullptr));
    if (form_out) *form_out = form;
    return PCF_OK;
}

// Validate, length-sort and pack one collection for a pairwise call; the
// keyed form also ranks its interval ends.
static cudaError_t prepare_pairwise(const pcf_csr* x, int form, Header* hdr, SetView& sv,
                                    const KeySort& ks, cudaStream_t s, bool auto64)
{
    KeyOut ko;
    if (form == kPackKeyed) { ko.key = ks.key[0]; ko.pay = ks.pay[0]; }
    cudaError_t e = prepare_set(x->offsets, x->times, x->values, x->dtype, x->n, x->nnz, true,
                                form, hdr, sv, s, form == kPackKeyed ? &ko : nullptr, auto64);
    if (e != cudaSuccess || form != kPackKeyed) return e;
    return rank_keys(ks, reinterpret_cast<KElem*>(sv.packed), sv.poff, x->n, nullptr, nullptr, 0,
                     hdr, s);
}

// Order keys of a window's bounds for a keyed walk (after the ranks exist).
static void keyed_bounds(WalkArgs& wa, const pcf_window* win, int form, const KeySort& ks,
                         KElem* pack0, KElem* pack1, Header* hdr, cudaStream_t s)
{
    if (form != kPackKeyed) return;
    const double lo = win ? win->a : 0.0;
    const double hi = win ? win->b : (double)INFINITY;
    split_time(lo, wa.lo_hl);
    split_time(hi, wa.hi_hl);
    if (lo > 0.0 || !std::isinf(hi)) {
        bound_keys(ks, pack0, pack1, lo, hi, hdr, s);
        wa.bound_keys = hdr->bound_key;
    } else {
        wa.bound_keys = nullptr;
    }
}

// Put the columns of matrices written with kOutRowsInputColsSorted back into
// the input order (the length sort's key buffer holds the inverse order).
// With s0 < s1 only the rows of sorted positions s0 .. s1 - 1, whose inverse
// order the caller has already computed.
static int finish_cols_sorted(const SetView& sv, const pcf_integral* F, int nF, int64_t n,
                              int out_f64, Header* hdr, cudaStream_t s, int64_t s0 = 0,
                              int64_t s1 = -1)
{
    uint32_t* pos = sv.khi[0];
    void* mats[PCF_MAX_INTEGRALS];
    for (int k = 0; k < nF; ++k) mats[k] = F[k].out;
    if (s1 < 0) {
        if (launch_inverse_perm(sv.perm, n, pos, hdr, s) != cudaSuccess ||
            launch_permute_cols(mats, nF, n, out_f64, pos, hdr, s) != cudaSuccess)
            return PCF_ECUDA;
        return PCF_OK;
    }
    if (launch_permute_cols(mats, nF, n, out_f64, pos, hdr, s, sv.perm, s0, s1) != cudaSuccess)
        return PCF_ECUDA;
    return PCF_OK;
}

int pcf_prepare(const pcf_csr* x, int precision, void* workspace, size_t workspace_bytes,
                cudaStream_t stream)
{
    if (!csr_ok(x)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    Header* hdr;
    SetView sv;
    KeySort ks;
    int form = kPackF64;
    int rc = pairwise_common(x, precision, workspace, workspace_bytes, &hdr, &sv, &ks, &form);
    if (rc != PCF_OK) return rc;
    init_header_kernel<<<1, 1, 0, stream>>>(hdr, 0);
    if (x->n == 0) return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
    if (prepare_pairwise(x, form, hdr, sv, ks, stream, pr.auto64) != cudaSuccess) return PCF_ECUDA;
    return PCF_OK;
}

int pcf_pairwise(const pcf_csr* x, const pcf_integral* F, int nF, int precision, int layout,
                 int out_dtype, int flags, void* workspace, size_t workspace_bytes,
                 cudaStream_t stream)
{
    return pcf_pairwise_ex(x, F, nF, precision, layout, out_dtype, flags, nullptr, nullptr,
                           workspace, workspace_bytes, stream);
}

int pcf_pairwise_ex(const pcf_csr* x, const pcf_integral* F, int nF, int precision, int layout,
                    int out_dtype, int flags, const pcf_schedule* schedule,
                    const pcf_window* window, void* workspace, size_t workspace_bytes,
                    cudaStream_t stream)
{
    if (!csr_ok(x)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    if (layout != PCF_OUT_FULL && layout != PCF_OUT_UPPER_PACKED && layout != PCF_OUT_FULL_SORTED)
        return PCF_EINVAL;
    if (out_dtype != PCF_F32 && out_dtype != PCF_F64) return PCF_EINVAL;
    if (flags & ~PCF_PAIRWISE_PREPARED) return PCF_EINVAL;
    if (check_schedule(schedule) != PCF_OK) return PCF_EINVAL;
    if (check_window(window) != PCF_OK) return PCF_EINVAL;
    int rc = check_requests(F, nF, x->n > 0);
    if (rc != PCF_OK) return rc;
    Header* hdr;
    SetView sv;
    KeySort ks;
    int form = kPackF64;
    rc = pairwise_common(x, precision, workspace, workspace_bytes, &hdr, &sv, &ks, &form);
    if (rc != PCF_OK) return rc;
    if (x->n == 0) return PCF_OK;
    if (!(flags & PCF_PAIRWISE_PREPARED)) {
        init_header_kernel<<<1, 1, 0, stream>>>(hdr, 0);
        if (prepare_pairwise(x, form, hdr, sv, ks, stream, pr.auto64) != cudaSuccess) return PCF_ECUDA;
    }

    WalkArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.pack_r = wa.pack_c = sv.packed;
    wa.poff_r = wa.poff_c = sv.poff;
    wa.slen_r = wa.slen_c = sv.slen;
    wa.perm_r = wa.perm_c = sv.perm;
    wa.n_r = wa.n_c = x->n;
    wa.nb_r = wa.nb_c = (x->n + kTile - 1) / kTile;
    wa.ntiles = wa.nb_r * (wa.nb_r + 1) / 2;
    wa.symmetric = 1;
    wa.hdr = hdr;
    wa.out_f64 = out_dtype == PCF_F64;
    wa.ld_out = x->n;
    // FULL matrices of one call (not a shard) whose rows fit the permutation
    // pass: written with sorted columns, then put back in place
    const bool cols_sorted = layout == PCF_OUT_FULL && !(schedule && schedule->shard_count > 1) &&
                             permute_cols_fits(x->n, wa.out_f64);
    wa.layout = cols_sorted ? kOutRowsInputColsSorted : layout;
    KElem* kp = reinterpret_cast<KElem*>(sv.packed);
    keyed_bounds(wa, window, form, ks, kp, kp, hdr, stream);
    rc = run_walks_for(wa, F, nF, pr, form, schedule, window, stream);
    if (rc != PCF_OK || !cols_sorted) return rc;
    return finish_cols_sorted(sv, F, nF, x->n, wa.out_f64, hdr, stream);
}

int pcf_pairwise_to_host(const pcf_csr* x, const pcf_integral* F, int nF, int precision,
                         int out_dtype, const pcf_schedule* schedule, void* const* host_out,
                         int nbands, void* workspace, size_t workspace_bytes,
                         cudaStream_t stream, cudaStream_t copy_stream)
{
    if (!csr_ok(x)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    if (out_dtype != PCF_F32 && out_dtype != PCF_F64) return PCF_EINVAL;
    if (nbands < 0) return PCF_EINVAL;
    if (check_schedule(schedule) != PCF_OK) return PCF_EINVAL;
    if (schedule && schedule->shard_count > 1) return PCF_EINVAL;
    int rc = check_requests(F, nF, x->n > 0);
    if (rc != PCF_OK) return rc;
    Header* hdr;
    SetView sv;
    KeySort ks;
    int form = kPackF64;
    rc = pairwise_common(x, precision, workspace, workspace_bytes, &hdr, &sv, &ks, &form);
    if (rc != PCF_OK) return rc;
    if (x->n == 0) return PCF_OK;
    if (!host_out) return PCF_EINVAL;
    RowCopy cp;
    memset(&cp, 0, sizeof cp);
    cp.n = nF;
    const int64_t N = x->n;
    const int64_t row_bytes = N * (out_dtype == PCF_F64 ? 8 : 4);
    bool vec16 = row_bytes % 16 == 0;
    for (int k = 0; k < nF; ++k) {
        void* dp = nullptr;
        if (!host_out[k] || cudaHostGetDevicePointer(&dp, host_out[k], 0) != cudaSuccess || !dp) {
            cudaGetLastError();   // the failed query's error is not sticky: clear it
            return PCF_EINVAL;
        }
        cp.src[k] = reinterpret_cast<const char*>(F[k].out);
        cp.dst[k] = reinterpret_cast<char*>(dp);
        vec16 = vec16 && (uintptr_t)cp.src[k] % 16 == 0 && (uintptr_t)cp.dst[k] % 16 == 0;
    }

    init_header_kernel<<<1, 1, 0, stream>>>(hdr, 0);
    if (prepare_pairwise(x, form, hdr, sv, ks, stream, pr.auto64) != cudaSuccess) return PCF_ECUDA;
    WalkArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.pack_r = wa.pack_c = sv.packed;
    wa.poff_r = wa.poff_c = sv.poff;
    wa.slen_r = wa.slen_c = sv.slen;
    wa.perm_r = wa.perm_c = sv.perm;
    wa.n_r = wa.n_c = N;
    wa.nb_r = wa.nb_c = (N + kTile - 1) / kTile;
    wa.ntiles = wa.nb_r * (wa.nb_r + 1) / 2;
    wa.symmetric = 1;
    wa.hdr = hdr;
    wa.out_f64 = out_dtype == PCF_F64;
    wa.ld_out = N;
    // rows written with sorted columns (whole DRAM sectors), gathered into the
    // input order by the copies; the device matrices are put back in place
    // after the last copy
    const bool cols_sorted = permute_cols_fits(N, wa.out_f64);
    wa.layout = cols_sorted ? kOutRowsInputColsSorted : PCF_OUT_FULL;
    uint32_t* pos = sv.khi[0];
    if (cols_sorted && launch_inverse_perm(sv.perm, N, pos, hdr, stream) != cudaSuccess)
        return PCF_ECUDA;
    {
        KElem* kp = reinterpret_cast<KElem*>(sv.packed);
        keyed_bounds(wa, nullptr, form, ks, kp, kp, hdr, stream);
    }
    const int sms = device_sm_count();
    const bool two = copy_stream != stream;
    // the walks run with the largest shared-memory carve-out; a CTA that asks
    // for another split of L1 cannot join an SM they occupy
    if (cudaFuncSetAttribute(copy_rows_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncSetAttribute(gather_rows_kernel<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncSetAttribute(gather_rows_kernel<double>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return PCF_ECUDA;

    // copies of sorted rows [s0, s1) once everything before on `stream` is done
    auto copy_rows = [&](int64_t s0, int64_t s1) -> bool {
        if (s1 <= s0) return true;
        cudaStream_t cs = stream;
        if (two) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return false;
            const bool ok = cudaEventRecord(ev, stream) == cudaSuccess &&
                            cudaStreamWaitEvent(copy_stream, ev, 0) == cudaSuccess;
            cudaEventDestroy(ev);
            if (!ok) return false;
            cs = copy_stream;
        }
        const int64_t cap = sms / 2 > 0 ? sms / 2 : 1;
        const int64_t grid = (s1 - s0) < cap ? (s1 - s0) : cap;
        if (!cols_sorted)
            copy_rows_kernel<<<(int)grid, 128, 0, cs>>>(cp, sv.perm, N, s0, s1, row_bytes,
                                                        vec16 ? 1 : 0, hdr);
        else if (wa.out_f64)
            gather_rows_kernel<double><<<(int)grid, 128, 0, cs>>>(cp, sv.perm, pos, N, s0, s1,
                                                                  vec16 ? 1 : 0, hdr);
        else
            gather_rows_kernel<float><<<(int)grid, 128, 0, cs>>>(cp, sv.perm, pos, N, s0, s1,
                                                                 vec16 ? 1 : 0, hdr);
        return cudaGetLastError() == cudaSuccess;
    };

    // the schedule, decided once for the whole matrix (a band alone is smaller)
    pcf_schedule sch;
    memset(&sch, 0, sizeof sch);
    if (schedule) sch = *schedule;
    if (sch.kernel == PCF_SCHED_AUTO)
        sch.kernel = wa.ntiles * 2 < sms ? PCF_SCHED_MERGEPATH : PCF_SCHED_TILE_1024;
    // `stream` continues after the last copy enqueued, also when a later
    // step fails (the caller may reuse the buffers after an error)
    auto join = [&]() -> bool {
        if (!two) return true;
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return false;
        const bool ok = cudaEventRecord(ev, copy_stream) == cudaSuccess &&
                        cudaStreamWaitEvent(stream, ev, 0) == cudaSuccess;
        cudaEventDestroy(ev);
        return ok;
    };
    auto fail = [&](int code) { join(); return code; };
    int64_t permuted = 0;   // sorted rows whose columns are back in the input order
    if (sch.kernel == PCF_SCHED_MERGEPATH || nbands == 1) {
        rc = run_walks_for(wa, F, nF, pr, form, &sch, nullptr, stream);
        if (rc != PCF_OK) return rc;
        if (!copy_rows(0, N)) return fail(PCF_ECUDA);
    } else {
        const int64_t units = (sch.kernel == PCF_SCHED_TILE_512X2 || sch.kernel == PCF_SCHED_TILE_512X3)
                                  ? 2 : 1;
        const int64_t NB = wa.nb_r;
        // first tile of row block m in the row order (row block i holds NB - i tiles)
        auto first_tile = [&](int64_t m) { return m * NB - m * (m - 1) / 2; };
        const std::vector<int64_t> cuts = plan_bands(NB, nbands == 0 ? 16 : nbands);
        wa.tile_order = 1;
        for (size_t k = 0; k + 1 < cuts.size(); ++k) {
            const int64_t m0 = cuts[k], m1 = cuts[k + 1];
            wa.ntiles = first_tile(m1);
            rc = run_walks_for(wa, F, nF, pr, form, &sch, nullptr, stream, first_tile(m0) * units);
            if (rc != PCF_OK) return fail(rc);
            const int64_t s0 = m0 * kTile;
            const int64_t s1 = m1 * kTile < N ? m1 * kTile : N;
            const bool last_band = k + 2 == cuts.size();
            cudaEvent_t copied = nullptr;    // the copies of the earlier bands
            if (last_band && cols_sorted && two) {
                if (cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventRecord(copied, copy_stream) != cudaSuccess) {
                    if (copied) cudaEventDestroy(copied);
                    return fail(PCF_ECUDA);
                }
            }
            if (!copy_rows(s0, s1)) {
                if (copied) cudaEventDestroy(copied);
                return fail(PCF_ECUDA);
            }
            if (copied) {
                // the device rows of the earlier bands are final and copied:
                // their columns go back to the input order while the last
                // band's rows are copied
                const bool ok = cudaStreamWaitEvent(stream, copied, 0) == cudaSuccess;
                cudaEventDestroy(copied);
                if (!ok) return fail(PCF_ECUDA);
                rc = finish_cols_sorted(sv, F, nF, N, wa.out_f64, hdr, stream, 0, s0);
                if (rc != PCF_OK) return fail(rc);
                permuted = s0;
            }
        }
    }
    if (!join()) return PCF_ECUDA;
    if (cols_sorted) {
        rc = permuted > 0 ? finish_cols_sorted(sv, F, nF, N, wa.out_f64, hdr, stream, permuted, N)
                          : finish_cols_sorted(sv, F, nF, N, wa.out_f64, hdr, stream);
        if (rc != PCF_OK) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
}

int pcf_cross(const pcf_csr* a, const pcf_csr* b, int64_t row_begin, int64_t row_end,
              const pcf_integral* F, int nF, int precision, int64_t ld_out, int out_dtype,
              int flags, void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    return pcf_cross_ex(a, b, row_begin, row_end, F, nF, precision, ld_out, out_dtype, flags,
                        nullptr, nullptr, workspace, workspace_bytes, stream);
}

// The cross walk of rows [row_begin, row_end) of a against b (checked
// arguments and workspace).  moved: a and b are collections built by earlier
// kernels of the call (moved to a weight's time): the header is already
// initialized, their offsets are not whole arrays and their validation is
// skipped after an earlier error.
static int cross_impl(const pcf_csr* a, const pcf_csr* b, int64_t row_begin, int64_t row_end,
                      const pcf_integral* F, int nF, const Prec& pr, int64_t ld_out, int out_dtype,
                      int flags, const pcf_schedule* schedule, const pcf_window* window,
                      void* workspace, cudaStream_t stream, bool moved)
{
    const int64_t rows = row_end - row_begin;
    const int form = call_form(pr, a, b);
    char* cur = (char*)workspace;
    Header* hdr = (Header*)cur;
    cur += sizeof(Header);
    const int es = call_elem_bytes(pr, form);
    SetView sb = carve_set(cur, b->n, b->nnz, es, 1);
    SetView sa = carve_set(cur, rows, a->nnz, es, 0);
    KeySort ks;
    if (form == kPackKeyed) ks = carve_keysort(cur, key_capacity(a, b));
    const bool reuse = (flags & PCF_CROSS_REUSE_B) != 0;
    if (!moved) init_header_kernel<<<1, 1, 0, stream>>>(hdr, reuse ? 1 : 0);
    // keyed: B's interval ends first in the sort input, then A's; both are
    // ranked together every call (A's rows change, so B's ranks do too: a
    // reused B keeps its validation and length sort and is packed again)
    KeyOut kb, ka;
    if (form == kPackKeyed) {
        kb.key = ka.key = ks.key[0];
        kb.pay = ka.pay = ks.pay[0];
        kb.set_bit = 0x80000000u;
        ka.base_poff = sb.poff;
        ka.base_n = b->n;
    }
    const KeyOut* pkb = form == kPackKeyed ? &kb : nullptr;
    const KeyOut* pka = form == kPackKeyed ? &ka : nullptr;
    const bool a64 = pr.auto64 && form != kPackF64;
    if (!reuse) {
        if (prepare_set(b->offsets, b->times, b->values, b->dtype, b->n, b->nnz, !moved, form, hdr,
                        sb, stream, pkb, a64, moved) != cudaSuccess)
            return PCF_ECUDA;
    }
    if (prepare_set(a->offsets + row_begin, a->times, a->values, a->dtype, rows, a->nnz,
                    !moved && row_begin == 0 && row_end == a->n, form, hdr, sa, stream, pka, a64,
                    moved) != cudaSuccess)
        return PCF_ECUDA;
    if (reuse && a64) {
        // the new rows may change the choice: B packed again in both gated forms
        if (pack_set(b->offsets, b->times, b->values, b->dtype, b->n, form, hdr, sb, stream, pkb,
                     &hdr->need64, 0) != cudaSuccess ||
            pack_set(b->offsets, b->times, b->values, b->dtype, b->n, kPackF64, hdr, sb, stream,
                     nullptr, &hdr->need64, 1) != cudaSuccess)
            return PCF_ECUDA;
    } else if (reuse && form == kPackKeyed) {
        if (pack_set(b->offsets, b->times, b->values, b->dtype, b->n, form, hdr, sb, stream, pkb) !=
            cudaSuccess)
            return PCF_ECUDA;
    }
    KElem* kpa = reinterpret_cast<KElem*>(sa.packed);
    KElem* kpb = reinterpret_cast<KElem*>(sb.packed);
    if (form == kPackKeyed &&
        rank_keys(ks, kpa, sa.poff, rows, kpb, sb.poff, b->n, hdr, stream) != cudaSuccess)
        return PCF_ECUDA;

    WalkArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.pack_r = sa.packed; wa.poff_r = sa.poff; wa.slen_r = sa.slen; wa.perm_r = sa.perm;
    wa.pack_c = sb.packed; wa.poff_c = sb.poff; wa.slen_c = sb.slen; wa.perm_c = sb.perm;
    wa.n_r = rows;
    wa.n_c = b->n;
    wa.nb_r = (rows + kTile - 1) / kTile;
    wa.nb_c = (b->n + kTile - 1) / kTile;
    wa.ntiles = wa.nb_r * wa.nb_c;
    wa.symmetric = 0;
    wa.hdr = hdr;
    wa.layout = PCF_OUT_FULL;
    wa.out_f64 = out_dtype == PCF_F64;
    wa.ld_out = ld_out;
    keyed_bounds(wa, window, form, ks, kpa, kpb, hdr, stream);
    return run_walks_for(wa, F, nF, pr, form, schedule, window, stream);
}

int pcf_cross_ex(const pcf_csr* a, const pcf_csr* b, int64_t row_begin, int64_t row_end,
                 const pcf_integral* F, int nF, int precision, int64_t ld_out, int out_dtype,
                 int flags, const pcf_schedule* schedule, const pcf_window* window,
                 void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    if (!csr_ok(a) || !csr_ok(b)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    if (out_dtype != PCF_F32 && out_dtype != PCF_F64) return PCF_EINVAL;
    if (row_begin < 0 || row_end < row_begin || row_end > a->n) return PCF_EINVAL;
    if (ld_out < b->n) return PCF_EINVAL;
    if (flags & ~PCF_CROSS_REUSE_B) return PCF_EINVAL;
    if (check_schedule(schedule) != PCF_OK) return PCF_EINVAL;
    if (check_window(window) != PCF_OK) return PCF_EINVAL;
    const int64_t rows = row_end - row_begin;
    int rc = check_requests(F, nF, rows > 0 && b->n > 0);
    if (rc != PCF_OK) return rc;
    const int form = call_form(pr, a, b);
    if (form == kPackKeyed && key_capacity(a, b) > 0x7fffffffLL) return PCF_EUNSUPPORTED;
    size_t need = 0;
    pcf_workspace_size(a, b, precision, PCF_WS_FORWARD, &need);
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || workspace_bytes < need) return PCF_ENOWS;
    if (rows == 0 || b->n == 0) return PCF_OK;
    return cross_impl(a, b, row_begin, row_end, F, nF, pr, ld_out, out_dtype, flags, schedule,
                      window, workspace, stream, false);
}

int pcf_pairwise_backward(const pcf_csr* x, int metric, double p, int apply_root,
                          const void* fwd_out, const void* grad_out, int grad_dtype,
                          void* grad_values, void* grad_times, void* workspace,
                          size_t workspace_bytes, cudaStream_t stream)
{
    return pcf_pairwise_backward_ex(x, metric, p, apply_root, fwd_out, grad_out, grad_dtype,
                                    grad_values, grad_times, nullptr, workspace, workspace_bytes,
                                    stream);
}

int pcf_pairwise_backward_ex(const pcf_csr* x, int metric, double p, int apply_root,
                             const void* fwd_out, const void* grad_out, int grad_dtype,
                             void* grad_values, void* grad_times, const pcf_schedule* schedule,
                             void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    if (!csr_ok(x)) return PCF_EINVAL;
    int64_t shard_index = 0, shard_count = 1;
    if (schedule) {
        for (int k = 0; k < 4; ++k)
            if (schedule->reserved[k]) return PCF_EINVAL;
        if (schedule->kernel != PCF_SCHED_AUTO && schedule->kernel != PCF_SCHED_TILE_1024)
            return PCF_EINVAL;
        if (schedule->shard_count > 1) {
            if (schedule->shard_index < 0 || schedule->shard_index >= schedule->shard_count)
                return PCF_EINVAL;
            shard_index = schedule->shard_index;
            shard_count = schedule->shard_count;
        } else if (schedule->shard_count < 0 || schedule->shard_index != 0) {
            return PCF_EINVAL;
        }
    }
    if (metric < PCF_L1 || metric > PCF_GRAM) return PCF_EINVAL;
    if (metric == PCF_LP && !(p >= 1.0 && std::isfinite(p))) return PCF_EINVAL;
    if (grad_dtype != PCF_F32 && grad_dtype != PCF_F64) return PCF_EINVAL;
    const double ex = metric == PCF_L1 ? 1.0 : metric == PCF_L2 ? 2.0 : metric == PCF_LP ? p : 1.0;
    const bool need_fwd = apply_root && metric != PCF_GRAM && ex != 1.0;
    if (x->n > 0 && (!grad_out || !grad_values || !grad_times)) return PCF_EINVAL;
    if (x->n > 0 && need_fwd && !fwd_out) return PCF_EINVAL;
    size_t need = 0;
    pcf_workspace_size(x, nullptr, PCF_PREC_F64, PCF_WS_BACKWARD, &need);
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || workspace_bytes < need) return PCF_ENOWS;
    if (x->n == 0) return PCF_OK;

    char* cur = (char*)workspace;
    Header* hdr = (Header*)cur;
    cur += sizeof(Header);
    SetView sv = carve_set(cur, x->n, x->nnz, 16, 0);
    double* gv = (double*)cur;
    cur += align_up(sizeof(double) * (size_t)x->nnz);
    double* gt = (double*)cur;
    init_header_kernel<<<1, 1, 0, stream>>>(hdr, 0);
    if (prepare_set(x->offsets, x->times, x->values, x->dtype, x->n, x->nnz, true, kPackF64, hdr,
                    sv, stream) != cudaSuccess)
        return PCF_ECUDA;
    {
        int64_t blocks = (x->nnz + 255) / 256;
        const int64_t cap = (int64_t)device_sm_count() * 16;
        if (blocks > cap) blocks = cap;
        zero_kernel<<<(int)blocks, 256, 0, stream>>>(gv, x->nnz);
        zero_kernel<<<(int)blocks, 256, 0, stream>>>(gt, x->nnz);
    }
    BackArgs ba;
    memset(&ba, 0, sizeof ba);
    ba.pack = (const double2*)sv.packed;
    ba.poff = sv.poff; ba.slen = sv.slen; ba.perm = sv.perm;
    ba.n = x->n;
    ba.nb = (x->n + kTile - 1) / kTile;
    ba.ntiles = ba.nb * (ba.nb + 1) / 2;
    ba.G = grad_out; ba.F = fwd_out; ba.g_f64 = grad_dtype == PCF_F64;
    ba.metric = metric; ba.p = p; ba.apply_root = apply_root ? 1 : 0;
    ba.gv = gv; ba.gt = gt; ba.hdr = hdr;
    ba.shard_index = shard_index; ba.shard_count = shard_count;
    if (launch_backward(ba, stream) != cudaSuccess) return PCF_ECUDA;
    if (launch_scatter_grad(sv, x->offsets, gv, gt, grad_values, grad_times,
                            x->dtype == PCF_F64, hdr, stream) != cudaSuccess)
        return PCF_ECUDA;
    return PCF_OK;
}

int pcf_segment_integrals(const pcf_csr* x, int functional, double p, int apply_root,
                          double a, double b, int precision, void* out, int out_dtype,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    if (!csr_ok(x)) return PCF_EINVAL;
    if (precision != PCF_PREC_F64 && precision != PCF_PREC_F32_COMP) return PCF_EINVAL;
    if (functional != PCF_FN_INTEGRAL && functional != PCF_FN_LP) return PCF_EINVAL;
    if (functional == PCF_FN_LP && !(p >= 1.0 && std::isfinite(p))) return PCF_EINVAL;
    if (!(a >= 0.0) || !(b > a) || std::isnan(b) || std::isinf(a)) return PCF_EINVAL;
    if (out_dtype != PCF_F32 && out_dtype != PCF_F64) return PCF_EINVAL;
    if (x->n > 0 && !out) return PCF_EINVAL;
    Header* hdr;
    SetView sv;
    int rc = pairwise_common(x, PCF_PREC_F64, workspace, workspace_bytes, &hdr, &sv);
    if (rc != PCF_OK) return rc;
    init_header_kernel<<<1, 1, 0, stream>>>(hdr, 0);
    if (x->n == 0) return cudaGetLastError() == cudaSuccess ? PCF_OK : PCF_ECUDA;
    // the input check runs inside the segment kernels (same reasons and indices)
    // scratch in the packed area: the chunk table and the long-PCF pieces
    // (60 bytes per chunk of 7,680 breakpoints, + 8; the area holds 16 per
    // breakpoint and at least 256)
    if (launch_segments(x, functional, p, apply_root, a, b, precision, out, out_dtype == PCF_F64,
                        hdr, sv.packed, stream) != cudaSuccess)
        return PCF_ECUDA;
    return PCF_OK;
}

int pcf_sort_order(const pcf_csr* x, int precision, const void* workspace,
                   size_t workspace_bytes, int32_t* perm_out, cudaStream_t stream)
{
    if (!csr_ok(x)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    if (x->n > 0 && !perm_out) return PCF_EINVAL;
    Header* hdr;
    SetView sv;
    int rc = pairwise_common(x, precision, const_cast<void*>(workspace), workspace_bytes, &hdr, &sv);
    if (rc != PCF_OK) return rc;
    if (x->n == 0) return PCF_OK;
    if (cudaMemcpyAsync(perm_out, sv.perm, sizeof(int32_t) * (size_t)x->n, cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
        return PCF_ECUDA;
    return PCF_OK;
}

int pcf_check(const void* workspace, cudaStream_t stream, int* detail, int64_t* index)
{
    if (!workspace) return PCF_ENOWS;
    unsigned long long key = 0;
    if (cudaMemcpyAsync(&key, workspace, sizeof key, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return PCF_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return PCF_ECUDA;
    if (key == kNoError) {
        if (detail) *detail = 0;
        if (index) *index = -1;
        return PCF_OK;
    }
    if (detail) *detail = (int)(key & 15ull);
    if (index) *index = (int64_t)((key >> 4) & ((1ull << 58) - 1));
    const int reason = (int)(key & 15ull);
    if (reason == kErrCapacity) return PCF_ENOWS;
    if (reason == kErrWait) return PCF_ETIMEOUT;
    return PCF_EINVAL;
}

// The collection x moved to the weighted time W(t): same PCF count, at most
// one breakpoint more per PCF, float64, offsets known on the device only.
static pcf_csr moved_shape(const pcf_csr* x)
{
    pcf_csr m;
    memset(&m, 0, sizeof m);
    m.n = x->n;
    m.nnz = x->nnz + x->n;
    m.dtype = PCF_F64;
    return m;
}

static bool weight_ok(const pcf_csr* w)
{
    return csr_ok(w) && w->n == 1 && w->nnz >= 1;
}

int pcf_weighted_workspace_size(const pcf_csr* x, const pcf_csr* w, int precision, size_t* bytes)
{
    if (!bytes || !x || x->n < 0 || x->nnz < 0 || x->n > 0x7fffffffLL) return PCF_EINVAL;
    if (!w || w->n != 1 || w->nnz < 1) return PCF_EINVAL;
    const pcf_csr m = moved_shape(x);
    size_t inner = 0;
    const int rc = pcf_workspace_size(&m, nullptr, precision, PCF_WS_FORWARD, &inner);
    if (rc != PCF_OK) return rc;
    *bytes = align_up(inner) + weight_scratch_bytes(x->n, x->nnz, w->nnz);
    return PCF_OK;
}

int pcf_pairwise_weighted(const pcf_csr* x, const pcf_csr* w, const pcf_integral* F, int nF,
                          int precision, int layout, int out_dtype, const pcf_schedule* schedule,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    if (!csr_ok(x) || !weight_ok(w)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    if (layout != PCF_OUT_FULL && layout != PCF_OUT_UPPER_PACKED && layout != PCF_OUT_FULL_SORTED)
        return PCF_EINVAL;
    if (out_dtype != PCF_F32 && out_dtype != PCF_F64) return PCF_EINVAL;
    if (check_schedule(schedule) != PCF_OK) return PCF_EINVAL;
    int rc = check_requests(F, nF, x->n > 0);
    if (rc != PCF_OK) return rc;
    size_t need = 0;
    rc = pcf_weighted_workspace_size(x, w, precision, &need);
    if (rc != PCF_OK) return rc;
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || workspace_bytes < need) return PCF_ENOWS;
    if (x->n == 0) return PCF_OK;

    // [the pairwise workspace of the moved collection][the weight scratch]
    pcf_csr m = moved_shape(x);
    size_t inner = 0;
    pcf_workspace_size(&m, nullptr, precision, PCF_WS_FORWARD, &inner);
    char* wcur = (char*)workspace + align_up(inner);
    const WeightScratch wsc = carve_weight(wcur, x->n, x->nnz, w->nnz);
    m.offsets = wsc.off2;
    m.times = wsc.t2;
    m.values = wsc.v2;
    Header* hdr;
    SetView sv;
    KeySort ks;
    int form = kPackF64;
    rc = pairwise_common(&m, precision, workspace, inner, &hdr, &sv, &ks, &form);
    if (rc != PCF_OK) return rc;

    init_header_kernel<<<1, 1, 0, stream>>>(hdr, 0);
    // x and w are checked before the moved collection is built from them
    if (launch_validate(x->offsets, x->times, x->values, x->dtype, x->n, x->nnz, kPackF64, hdr, sv,
                        stream) != cudaSuccess ||
        launch_weight_move(x, w, wsc, hdr, stream) != cudaSuccess)
        return PCF_ECUDA;
    KeyOut ko;
    if (form == kPackKeyed) { ko.key = ks.key[0]; ko.pay = ks.pay[0]; }
    if (prepare_set(m.offsets, m.times, m.values, PCF_F64, m.n, m.nnz, false, form, hdr, sv, stream,
                    form == kPackKeyed ? &ko : nullptr, pr.auto64, true) != cudaSuccess)
        return PCF_ECUDA;
    if (form == kPackKeyed &&
        rank_keys(ks, reinterpret_cast<KElem*>(sv.packed), sv.poff, m.n, nullptr, nullptr, 0, hdr,
                  stream) != cudaSuccess)
        return PCF_ECUDA;

    WalkArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.pack_r = wa.pack_c = sv.packed;
    wa.poff_r = wa.poff_c = sv.poff;
    wa.slen_r = wa.slen_c = sv.slen;
    wa.perm_r = wa.perm_c = sv.perm;
    wa.n_r = wa.n_c = m.n;
    wa.nb_r = wa.nb_c = (m.n + kTile - 1) / kTile;
    wa.ntiles = wa.nb_r * (wa.nb_r + 1) / 2;
    wa.symmetric = 1;
    wa.hdr = hdr;
    wa.out_f64 = out_dtype == PCF_F64;
    wa.ld_out = m.n;
    const bool cols_sorted = layout == PCF_OUT_FULL && !(schedule && schedule->shard_count > 1) &&
                             permute_cols_fits(m.n, wa.out_f64);
    wa.layout = cols_sorted ? kOutRowsInputColsSorted : layout;
    KElem* kp = reinterpret_cast<KElem*>(sv.packed);
    keyed_bounds(wa, nullptr, form, ks, kp, kp, hdr, stream);
    rc = run_walks_for(wa, F, nF, pr, form, schedule, nullptr, stream);
    if (rc != PCF_OK || !cols_sorted) return rc;
    return finish_cols_sorted(sv, F, nF, m.n, wa.out_f64, hdr, stream);
}

// Shapes of a cross call against a weight: rows [row_begin, row_end) of a
// and all of b, each moved to W(t).
static void cross_moved_shapes(const pcf_csr* a, const pcf_csr* b, int64_t rows, pcf_csr* am,
                               pcf_csr* bm)
{
    pcf_csr ar = *a;
    ar.n = rows;
    *am = moved_shape(&ar);
    *bm = moved_shape(b);
}

int pcf_cross_weighted_workspace_size(const pcf_csr* a, const pcf_csr* b, const pcf_csr* w,
                                      int precision, size_t* bytes)
{
    if (!bytes || !a || !b || a->n < 0 || b->n < 0 || a->nnz < 0 || b->nnz < 0 ||
        a->n > 0x7fffffffLL || b->n > 0x7fffffffLL)
        return PCF_EINVAL;
    if (!w || w->n != 1 || w->nnz < 1) return PCF_EINVAL;
    pcf_csr am, bm;
    cross_moved_shapes(a, b, a->n, &am, &bm);
    size_t inner = 0;
    const int rc = pcf_workspace_size(&am, &bm, precision, PCF_WS_FORWARD, &inner);
    if (rc != PCF_OK) return rc;
    *bytes = align_up(inner) + weight_scratch_bytes(a->n, a->nnz, w->nnz) +
             weight_scratch_bytes(b->n, b->nnz, w->nnz);
    return PCF_OK;
}

int pcf_cross_weighted(const pcf_csr* a, const pcf_csr* b, int64_t row_begin, int64_t row_end,
                       const pcf_csr* w, const pcf_integral* F, int nF, int precision,
                       int64_t ld_out, int out_dtype, const pcf_schedule* schedule,
                       void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    if (!csr_ok(a) || !csr_ok(b) || !weight_ok(w)) return PCF_EINVAL;
    Prec pr;
    if (!parse_prec(precision, &pr)) return PCF_EINVAL;
    if (out_dtype != PCF_F32 && out_dtype != PCF_F64) return PCF_EINVAL;
    if (row_begin < 0 || row_end < row_begin || row_end > a->n) return PCF_EINVAL;
    if (ld_out < b->n) return PCF_EINVAL;
    if (check_schedule(schedule) != PCF_OK) return PCF_EINVAL;
    const int64_t rows = row_end - row_begin;
    int rc = check_requests(F, nF, rows > 0 && b->n > 0);
    if (rc != PCF_OK) return rc;
    size_t need = 0;
    rc = pcf_cross_weighted_workspace_size(a, b, w, precision, &need);
    if (rc != PCF_OK) return rc;
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || workspace_bytes < need) return PCF_ENOWS;
    if (rows == 0 || b->n == 0) return PCF_OK;

    // [the cross workspace of the moved collections][weight scratch a][b]
    pcf_csr am, bm, afull;
    cross_moved_shapes(a, b, a->n, &am, &afull);
    cross_moved_shapes(a, b, rows, &am, &bm);
    size_t inner = 0;
    {
        pcf_csr am_full = moved_shape(a);
        pcf_workspace_size(&am_full, &bm, precision, PCF_WS_FORWARD, &inner);
    }
    char* wcur = (char*)workspace + align_up(inner);
    const WeightScratch wa_s = carve_weight(wcur, rows, a->nnz, w->nnz);
    const WeightScratch wb_s = carve_weight(wcur, b->n, b->nnz, w->nnz);
    am.offsets = wa_s.off2; am.times = wa_s.t2; am.values = wa_s.v2;
    bm.offsets = wb_s.off2; bm.times = wb_s.t2; bm.values = wb_s.v2;
    const int form = call_form(pr, &am, &bm);
    if (form == kPackKeyed && key_capacity(&am, &bm) > 0x7fffffffLL) return PCF_EUNSUPPORTED;

    Header* hdr = (Header*)workspace;
    init_header_kernel<<<1, 1, 0, stream>>>(hdr, 0);
    // the inputs are checked before they are moved (scratch set views of the
    // cross workspace serve the checks' length arrays)
    {
        char* cur = (char*)workspace + sizeof(Header);
        SetView sb = carve_set(cur, bm.n, bm.nnz, call_elem_bytes(pr, form), 1);
        SetView sa = carve_set(cur, rows, am.nnz, call_elem_bytes(pr, form), 0);
        pcf_csr arows = *a;
        arows.offsets = a->offsets + row_begin;
        arows.n = rows;
        if (launch_validate(b->offsets, b->times, b->values, b->dtype, b->n, b->nnz, kPackF64, hdr,
                            sb, stream) != cudaSuccess ||
            launch_validate(arows.offsets, a->times, a->values, a->dtype, rows, a->nnz, kPackF64,
                            hdr, sa, stream, row_begin == 0 && row_end == a->n) != cudaSuccess ||
            launch_weight_move(&arows, w, wa_s, hdr, stream) != cudaSuccess ||
            launch_weight_move(b, w, wb_s, hdr, stream) != cudaSuccess)
            return PCF_ECUDA;
    }
    return cross_impl(&am, &bm, 0, rows, F, nF, pr, ld_out, out_dtype, 0, schedule, nullptr,
                      workspace, stream, true);
}

int pcf_walk_promoted(const void* workspace, cudaStream_t stream, int* promoted)
{
    if (!workspace || !promoted) return PCF_EINVAL;
    unsigned int need = 0;
    const char* w = static_cast<const char*>(workspace);
    if (cudaMemcpyAsync(&need, w + offsetof(Header, need64), sizeof need, cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess)
        return PCF_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return PCF_ECUDA;
    *promoted = need != 0u ? 1 : 0;
    return PCF_OK;
}

const char* pcf_status_string(int status)
{
    switch (status) {
    case PCF_OK: return "ok";
    case PCF_EINVAL: return "invalid argument or invalid PCF data";
    case PCF_ENOWS: return "workspace missing, misaligned or too small";
    case PCF_ECUDA: return "CUDA runtime error";
    case PCF_ETIMEOUT: return "bounded device wait gave up";
    case PCF_EUNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

const char* pcf_version(void) { return "pcf_gb300 1 sm_103a"; }

}  // extern "C"
