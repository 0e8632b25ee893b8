// backward.cu -- adjoint of L = sum_{i,j} G_ij F_ij over the pairwise matrix.
//
// Not in the paper (Sec. 3 only remarks that derivatives of a parametrised
// antiderivative are available).  Differentiating each rectangle term
// h(v_f, v_g) (r - l) of Eq. simpleint:
//   d/dv_f  of the rectangle = dh/da(v_f, v_g) (r - l)       (value gradient)
//   d/dt_k  where f moves from v_{k-1} to v_k at t_k
//           = h(v_{k-1}, g(t_k-)) - h(v_k, g(t_k-))           (time gradient)
// with g(t_k-) the value of g just before t_k (left derivative where both PCFs
// share the breakpoint).  The walk is recomputed per pair in float64 with the
// simultaneous advance of Alg. 1, which hands both sides the pre-advance
// values at a shared breakpoint.  A multi-GPU split walks only the tiles t
// with t % shard_count == shard_index; the partial gradients of all shards
// sum to the whole (one all-reduce).  Each unordered pair i < j is walked once
// with weight (G_ij + G_ji) r'(I_ij); the Gram diagonal F_ii = int f_i^2 is
// differentiated by segment iteration (Sec. 3.2, Alg. 3).  Contributions are
// summed with float64 atomics into packed-order accumulators, then scattered
// back to the input order.
#include <cmath>

#include "internal.cuh"

namespace pcfgb {

template <int METRIC>
__device__ __forceinline__ double bw_h(double a, double b, double p)
{
    const double d = a - b;
    if constexpr (METRIC == PCF_L1) return fabs(d);
    else if constexpr (METRIC == PCF_L2) return d * d;
    else if constexpr (METRIC == PCF_LP) {
        if (p == 3.0) { double ad = fabs(d); return ad * ad * ad; }
        return pow(fabs(d), p);
    }
    else return a * b;
}

template <int METRIC>
__device__ __forceinline__ double bw_dh(double a, double b, double p)
{
    const double d = a - b;
    const double s = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
    if constexpr (METRIC == PCF_L1) return s;
    else if constexpr (METRIC == PCF_L2) return 2.0 * d;
    else if constexpr (METRIC == PCF_LP) {
        if (d == 0.0) return 0.0;
        const double e = p - 1.0;
        double ad = fabs(d), q;
        if (e == 1.0) q = ad;
        else if (e == 2.0) q = ad * ad;
        else q = pow(ad, e);
        return p * q * s;
    }
    else return b;
}

__device__ __forceinline__ double exponent_of(int metric, double p)
{
    return metric == PCF_L1 ? 1.0 : metric == PCF_L2 ? 2.0 : metric == PCF_LP ? p : 1.0;
}

__device__ __forceinline__ double load_mat(const void* m, int f64, int64_t idx)
{
    return f64 ? reinterpret_cast<const double*>(m)[idx] : (double)reinterpret_cast<const float*>(m)[idx];
}

template <int METRIC>
__global__ void __launch_bounds__(1024) backward_kernel(const BackArgs a)
{
    if (a.hdr->err != kNoError) return;
    const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
    const int64_t NB = a.nb;
    for (int64_t u = blockIdx.x;; u += gridDim.x) {
        const int64_t t = a.shard_index + u * a.shard_count;   // this shard's tiles
        if (t >= a.ntiles) break;
        // the forward walk's upper-triangle tile order (row block bi <= column block bj)
        int64_t bi, bj;
        decode_upper_tile(NB, t, 0, bi, bj);
        const int64_t gi = bi * kTile + r, gj = bj * kTile + c;
        if (gi >= a.n || gj >= a.n) continue;
        if (bi == bj && r > c) continue;
        const int64_t i = a.perm[gi], j = a.perm[gj];
        const int64_t of = a.poff[gi], og = a.poff[gj];
        const int nf = a.slen[gi];

        if (gi == gj) {
            if (METRIC != PCF_GRAM) continue;
            // Gram diagonal: both arguments move together (segment iteration)
            const double w = load_mat(a.G, a.g_f64, i * a.n + i);
            double tprev = 0.0, vprev = 0.0;
            for (int k = 0; k < nf; ++k) {
                const double2 e = a.pack[of + k];
                const double len = e.x - tprev;
                double gv;
                if (isinf(e.x)) gv = (e.y != 0.0) ? w * 2.0 * e.y * INFINITY : 0.0;
                else gv = w * 2.0 * e.y * len;
                atomicAdd(&a.gv[of + k], gv);
                if (k >= 1) atomicAdd(&a.gt[of + k], w * (vprev * vprev - e.y * e.y));
                tprev = e.x;
                vprev = e.y;
            }
            continue;
        }

        double w = load_mat(a.G, a.g_f64, i * a.n + j) + load_mat(a.G, a.g_f64, j * a.n + i);
        const double ex = exponent_of(METRIC, a.p);
        if (a.apply_root && METRIC != PCF_GRAM && ex != 1.0) {
            const double F = load_mat(a.F, a.g_f64, i * a.n + j);
            if (F == 0.0) continue;
            w *= (1.0 / ex) * pow(F, 1.0 - ex);    // r'(I) with I = F^ex
        }
        if (w == 0.0) continue;

        // Alg. 1 walk over [0, inf) with simultaneous advance on ties.  End
        // times are compared by their bit patterns on the integer pipe
        // (non-negative doubles order like their bits; +inf marks the tail).
        // For L1, L2 and the Gram the value gradients of both sides share one
        // product, and the time gradient h(v_old, g) - h(v_new, g) is taken
        // in factored form; every integrand is symmetric, h(a, b) = h(b, a),
        // so the side that advances (f on a tie) is handled by one
        // branch-free update with selected operands and addresses -- lanes
        // of a warp advancing different sides no longer run two half-empty
        // branches -- and the second side of a shared breakpoint by a rare
        // extra branch.  float64 operations per rectangle: L2 9, Gram 7, L1 7.
        int kf = 0, kg = 0;
        double2 ef = a.pack[of], eg = a.pack[og];
        double tc = 0.0, gvf = 0.0, gvg = 0.0;
        const long long kInfBits = 0x7ff0000000000000ll;
        const double w2 = 2.0 * w;
        for (;;) {
            const long long bf = __double_as_longlong(ef.x), bg = __double_as_longlong(eg.x);
            const bool sf = bf <= bg;               // f advances (also on a tie)
            const long long bn = sf ? bf : bg;
            if (bn == kInfBits) break;
            const bool tie = bf == bg;
            const double tn = __longlong_as_double(bn);
            const double dt = tn - tc;
            const double vf = ef.y, vg = eg.y;
            const int64_t at = sf ? of + kf : og + kg;   // advancing side's current element
            const double2 nx = a.pack[at + 1];
            const double v_old = sf ? vf : vg, other = sf ? vg : vf;
            double d = 0.0;
            if constexpr (METRIC == PCF_L2) {
                // dh/dv_f = 2 d = -dh/dv_g
                d = vf - vg;
                const double e = d * dt;
                gvf = fma(w2, e, gvf);
                gvg = fma(-w2, e, gvg);
            } else if constexpr (METRIC == PCF_GRAM) {
                // dh/dv_f = v_g, dh/dv_g = v_f
                const double wdt = w * dt;
                gvf = fma(wdt, vg, gvf);
                gvg = fma(wdt, vf, gvg);
            } else if constexpr (METRIC == PCF_L1) {
                // dh/dv_f = sign(d) = -dh/dv_g, 0 where d = 0
                d = vf - vg;
                const long long db = __double_as_longlong(d);
                const double wdt = w * dt;
                const double sw = (db << 1) == 0 ? 0.0 : (db < 0 ? -wdt : wdt);
                gvf += sw;
                gvg -= sw;
            } else {
                gvf += w * bw_dh<METRIC>(vf, vg, a.p) * dt;
                gvg += w * bw_dh<METRIC>(vg, vf, a.p) * dt;
            }
            // h(v_old, other) - h(v_new, other) for the advancing side
            auto tgrad = [&](double vo, double vn, double ot) -> double {
                if constexpr (METRIC == PCF_L2) { const double bb = vn - ot; return fma(d, d, -(bb * bb)); }
                else if constexpr (METRIC == PCF_GRAM) return (vo - vn) * ot;
                else if constexpr (METRIC == PCF_L1) return fabs(d) - fabs(vn - ot);
                else return bw_h<METRIC>(vo, ot, a.p) - bw_h<METRIC>(vn, ot, a.p);
            };
            atomicAdd(&a.gv[at], sf ? gvf : gvg);
            atomicAdd(&a.gt[at + 1], w * tgrad(v_old, nx.y, other));
            if (sf) { gvf = 0.0; ++kf; ef = nx; } else { gvg = 0.0; ++kg; eg = nx; }
            if (tie) {
                // shared breakpoint: g advances too, against f's value before it
                const double2 ng = a.pack[og + kg + 1];
                atomicAdd(&a.gv[og + kg], gvg);
                atomicAdd(&a.gt[og + kg + 1], w * tgrad(vg, ng.y, vf));
                gvg = 0.0;
                ++kg;
                eg = ng;
            }
            tc = tn;
        }
        // tail [t_last, inf): infinite width, finite only where dh = 0
        const double df = bw_dh<METRIC>(ef.y, eg.y, a.p), dg = bw_dh<METRIC>(eg.y, ef.y, a.p);
        if (df != 0.0) gvf += w * df * INFINITY;
        if (dg != 0.0) gvg += w * dg * INFINITY;
        atomicAdd(&a.gv[of + kf], gvf);
        atomicAdd(&a.gv[og + kg], gvg);
    }
}

// One warp per sorted PCF: packed-order accumulators -> caller's input order.
__global__ void scatter_grad_kernel(const int64_t* __restrict__ offsets, const int32_t* __restrict__ perm,
                                    const int32_t* __restrict__ slen, const int64_t* __restrict__ poff,
                                    int64_t n, const double* __restrict__ gv, const double* __restrict__ gt,
                                    void* grad_values, void* grad_times, int out_f64, const Header* hdr)
{
    if (hdr->err != kNoError) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp0; s < n; s += nwarps) {
        const int64_t o = offsets[perm[s]];
        const int64_t src = poff[s];
        const int len = slen[s];
        for (int k = lane; k < len; k += 32) {
            const double v = gv[src + k];
            const double t = (k == 0) ? 0.0 : gt[src + k];
            if (out_f64) {
                reinterpret_cast<double*>(grad_values)[o + k] = v;
                reinterpret_cast<double*>(grad_times)[o + k] = t;
            } else {
                reinterpret_cast<float*>(grad_values)[o + k] = (float)v;
                reinterpret_cast<float*>(grad_times)[o + k] = (float)t;
            }
        }
    }
}

cudaError_t launch_backward(const BackArgs& a, cudaStream_t s)
{
    if (a.ntiles <= a.shard_index) return cudaSuccess;
    int64_t grid = (a.ntiles - a.shard_index + a.shard_count - 1) / a.shard_count;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (grid > cap) grid = cap;
    switch (a.metric) {
    case PCF_L1: backward_kernel<PCF_L1><<<(int)grid, 1024, 0, s>>>(a); break;
    case PCF_L2: backward_kernel<PCF_L2><<<(int)grid, 1024, 0, s>>>(a); break;
    case PCF_LP: backward_kernel<PCF_LP><<<(int)grid, 1024, 0, s>>>(a); break;
    default: backward_kernel<PCF_GRAM><<<(int)grid, 1024, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_grad(const SetView& sv, const int64_t* offsets, const double* gv,
                                const double* gt, void* grad_values, void* grad_times,
                                int out_f64, Header* hdr, cudaStream_t s)
{
    if (sv.n == 0) return cudaSuccess;
    int64_t blocks = (sv.n * 32 + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    scatter_grad_kernel<<<(int)blocks, 256, 0, s>>>(offsets, sv.perm, sv.slen, sv.poff, sv.n, gv, gt,
                                                     grad_values, grad_times, out_f64, hdr);
    return cudaGetLastError();
}

}  // namespace pcfgb
