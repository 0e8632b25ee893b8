// weight.cu -- integrals against a non-negative PCF weight w: int h(f, g) w dt.
//
// The weighted L_p distance of Sec. 2.2 (the weight multiplying |f - g|^p)
// and the weighted inner product are combination integrals whose integrand
// depends on time through w.  With W(t) = int_0^t w, the antiderivative form
// of Sec. 3 gives each rectangle [l, r) of the pair walk the contribution
// h(f, g) * (W(r) - W(l)), and W is piecewise linear with its kinks at w's
// breakpoints.  So the weighted matrices are the unweighted matrices of the
// collection whose breakpoints are moved to s_k = W(t_k): every pair walk of
// the moved collection visits the same rectangles, each with width
// W(r) - W(l).  The kernels here build that collection once per call:
//
//   weight_scan_kernel   one CTA: checks w (values >= 0) and writes
//                        W at w's breakpoints by an ordered prefix sum
//   weight_count_kernel  warp per PCF: s_k = W(t_k) by binary search in w's
//                        breakpoints; an interval [s_k, s_{k+1}) of zero
//                        width (w = 0 on [t_k, t_{k+1})) is dropped; when w
//                        ends with value 0, W(inf) is finite and every PCF
//                        gets a last breakpoint at W(inf) with value 0, so
//                        the tail beyond the weight's support adds nothing;
//                        writes the new lengths
//   weight_scan_offsets_kernel  one CTA: offsets of the new collection
//   weight_write_kernel  warp per PCF: the kept breakpoints, compacted
//
// The moved collection is float64 (times and values); its walk is any of the
// library's walks (float32 ones compare its float64 times exactly).
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace pcfgb {

// W at w's breakpoints: Wt[k] = sum_{j < k} vw[j] (tw[j+1] - tw[j]) in a
// fixed order (thread chunks, then the chunk sums), so the result does not
// depend on scheduling.  Also checks w: offsets {0, nw}, t_0 = 0, times
// finite and increasing, values finite and >= 0 (reason 10 at the element).
template <typename T>
__global__ void __launch_bounds__(256) weight_scan_kernel(const int64_t* __restrict__ ow,
                                                          const T* __restrict__ tw,
                                                          const T* __restrict__ vw, int64_t nw,
                                                          double* __restrict__ Wt, Header* hdr)
{
    __shared__ double csum[256];
    const int tid = threadIdx.x;
    if (tid == 0 && (ow[0] != 0 || ow[1] != nw)) record_error(hdr, kErrWeight, 0);
    const int64_t chunk = (nw + 255) / 256;
    const int64_t b0 = (int64_t)tid * chunk;
    const int64_t b1 = b0 + chunk < nw ? b0 + chunk : nw;
    double s = 0.0;
    for (int64_t k = b0; k < b1; ++k) {
        const double v = (double)vw[k], t = (double)tw[k];
        const bool ok = v >= 0.0 && v <= DBL_MAX && t <= DBL_MAX &&
                        (k == 0 ? t == 0.0 : t > (double)tw[k - 1]);
        if (!ok) record_error(hdr, kErrWeight, k);
        if (k + 1 < nw) s += v * ((double)tw[k + 1] - t);
    }
    csum[tid] = s;
    __syncthreads();
    if (tid == 0) {
        double run = 0.0;
        for (int c = 0; c < 256; ++c) {
            const double x = csum[c];
            csum[c] = run;
            run += x;
        }
    }
    __syncthreads();
    double run = csum[tid];
    for (int64_t k = b0; k < b1; ++k) {
        Wt[k] = run;
        if (k + 1 < nw) run += (double)vw[k] * ((double)tw[k + 1] - (double)tw[k]);
    }
}

// W(t) for t >= 0: the last weight breakpoint tw[j] <= t, then the linear
// piece W[j] + vw[j] (t - tw[j]).
template <typename T>
__device__ __forceinline__ double weight_at(const T* __restrict__ tw, const T* __restrict__ vw,
                                            const double* __restrict__ Wt, int64_t nw, double t)
{
    int64_t lo = 0, hi = nw - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((double)tw[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return Wt[lo] + (double)vw[lo] * (t - (double)tw[lo]);
}

// For breakpoint k of a PCF with n breakpoints: is its interval kept?  An
// interval of zero moved width is dropped; the last interval is kept unless
// a finite W(inf) closes it with zero width (the added last breakpoint takes
// its place).
__device__ __forceinline__ bool weight_keep(int64_t k, int64_t n, double sk, double sk1,
                                            bool finite_end, double Winf)
{
    if (k + 1 < n) return sk < sk1;
    return finite_end ? sk < Winf : true;
}

template <typename Tx, typename Tw>
__global__ void weight_count_kernel(const int64_t* __restrict__ offsets, const Tx* __restrict__ times,
                                    int64_t n, const Tw* __restrict__ tw, const Tw* __restrict__ vw,
                                    const double* __restrict__ Wt, int64_t nw,
                                    int64_t* __restrict__ lens2, const Header* hdr)
{
    if (hdr->err != kNoError) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool finite_end = (double)vw[nw - 1] == 0.0;
    const double Winf = Wt[nw - 1];
    for (int64_t i = warp0; i < n; i += nwarps) {
        const int64_t o0 = offsets[i], o1 = offsets[i + 1], len = o1 - o0;
        int64_t kept = 0;
        for (int64_t k = lane; k < len; k += 32) {
            const double sk = weight_at(tw, vw, Wt, nw, (double)times[o0 + k]);
            const double sk1 = k + 1 < len ? weight_at(tw, vw, Wt, nw, (double)times[o0 + k + 1]) : 0.0;
            kept += weight_keep(k, len, sk, sk1, finite_end, Winf) ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
        if (lane == 0) lens2[i] = kept + (finite_end ? 1 : 0);
    }
}

// Exclusive scan of the new lengths into offsets (one CTA, fixed order).
__global__ void __launch_bounds__(1024) weight_scan_offsets_kernel(const int64_t* __restrict__ lens2,
                                                                   int64_t n,
                                                                   int64_t* __restrict__ off2,
                                                                   const Header* hdr)
{
    __shared__ int64_t csum[1024];
    if (hdr->err != kNoError) return;
    const int tid = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b0 = (int64_t)tid * chunk;
    const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += lens2[i];
    csum[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int c = 0; c < 1024; ++c) {
            const int64_t x = csum[c];
            csum[c] = run;
            run += x;
        }
        off2[n] = run;
    }
    __syncthreads();
    int64_t run = csum[tid];
    for (int64_t i = b0; i < b1; ++i) {
        off2[i] = run;
        run += lens2[i];
    }
}

template <typename Tx, typename Tw>
__global__ void weight_write_kernel(const int64_t* __restrict__ offsets, const Tx* __restrict__ times,
                                    const Tx* __restrict__ values, int64_t n,
                                    const Tw* __restrict__ tw, const Tw* __restrict__ vw,
                                    const double* __restrict__ Wt, int64_t nw,
                                    const int64_t* __restrict__ off2, double* __restrict__ t2,
                                    double* __restrict__ v2, const Header* hdr)
{
    if (hdr->err != kNoError) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool finite_end = (double)vw[nw - 1] == 0.0;
    const double Winf = Wt[nw - 1];
    for (int64_t i = warp0; i < n; i += nwarps) {
        const int64_t o0 = offsets[i], o1 = offsets[i + 1], len = o1 - o0;
        int64_t pos = off2[i];
        for (int64_t base = 0; base < len; base += 32) {
            const int64_t k = base + lane;
            bool keep = false;
            double sk = 0.0;
            if (k < len) {
                sk = weight_at(tw, vw, Wt, nw, (double)times[o0 + k]);
                const double sk1 = k + 1 < len ? weight_at(tw, vw, Wt, nw, (double)times[o0 + k + 1]) : 0.0;
                keep = weight_keep(k, len, sk, sk1, finite_end, Winf);
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int64_t q = pos + __popc(m & ((1u << lane) - 1u));
                t2[q] = sk;
                v2[q] = (double)values[o0 + k];
            }
            pos += __popc(m);
        }
        if (finite_end && lane == 0) {
            t2[pos] = Winf;
            v2[pos] = 0.0;
        }
    }
}

static int grid_warps(int64_t warps)
{
    int64_t blocks = (warps * 32 + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <typename Tx, typename Tw>
static cudaError_t launch_move(const pcf_csr* x, const pcf_csr* w, const WeightScratch& ws,
                               Header* hdr, cudaStream_t s)
{
    const Tw* tw = (const Tw*)w->times;
    const Tw* vw = (const Tw*)w->values;
    const int g = grid_warps(x->n);
    weight_count_kernel<Tx, Tw><<<g, 256, 0, s>>>(x->offsets, (const Tx*)x->times, x->n, tw, vw,
                                                  ws.Wt, w->nnz, ws.lens2, hdr);
    weight_scan_offsets_kernel<<<1, 1024, 0, s>>>(ws.lens2, x->n, ws.off2, hdr);
    weight_write_kernel<Tx, Tw><<<g, 256, 0, s>>>(x->offsets, (const Tx*)x->times,
                                                  (const Tx*)x->values, x->n, tw, vw, ws.Wt,
                                                  w->nnz, ws.off2, ws.t2, ws.v2, hdr);
    return cudaGetLastError();
}

cudaError_t launch_weight_move(const pcf_csr* x, const pcf_csr* w, const WeightScratch& ws,
                               Header* hdr, cudaStream_t s)
{
    if (w->dtype == PCF_F64)
        weight_scan_kernel<double><<<1, 256, 0, s>>>(w->offsets, (const double*)w->times,
                                                     (const double*)w->values, w->nnz, ws.Wt, hdr);
    else
        weight_scan_kernel<float><<<1, 256, 0, s>>>(w->offsets, (const float*)w->times,
                                                    (const float*)w->values, w->nnz, ws.Wt, hdr);
    if (x->dtype == PCF_F64)
        return w->dtype == PCF_F64 ? launch_move<double, double>(x, w, ws, hdr, s)
                                   : launch_move<double, float>(x, w, ws, hdr, s);
    return w->dtype == PCF_F64 ? launch_move<float, double>(x, w, ws, hdr, s)
                               : launch_move<float, float>(x, w, ws, hdr, s);
}

size_t weight_scratch_bytes(int64_t n, int64_t nnz, int64_t nw)
{
    return align_up(sizeof(double) * (size_t)(nw > 0 ? nw : 1)) +
           align_up(sizeof(int64_t) * (size_t)(n + 1)) * 2 +
           2 * align_up(sizeof(double) * (size_t)(nnz + n));
}

WeightScratch carve_weight(char*& cur, int64_t n, int64_t nnz, int64_t nw)
{
    WeightScratch w;
    auto take = [&](size_t bytes) { char* p = cur; cur += align_up(bytes); return p; };
    w.Wt = reinterpret_cast<double*>(take(sizeof(double) * (size_t)(nw > 0 ? nw : 1)));
    w.lens2 = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)(n + 1)));
    w.off2 = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * (size_t)(n + 1)));
    w.t2 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)(nnz + n)));
    w.v2 = reinterpret_cast<double*>(take(sizeof(double) * (size_t)(nnz + n)));
    w.cap = nnz + n;
    return w;
}

}  // namespace pcfgb
