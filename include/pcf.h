/*
 * pcf.h -- C ABI of the GB300 (sm_103a) PCF integral-matrix library.
 *
 * A piecewise constant function (PCF) f on [0, inf) is given by breakpoints
 * 0 = t_0 < t_1 < ... < t_{n-1} and values v_0..v_{n-1}; f = v_k on
 * [t_k, t_{k+1}) and f = v_{n-1} on [t_{n-1}, inf) (Sec. 2, PCF definition
 * and its n x 2 matrix storage).  A collection of N PCFs is passed in CSR form
 * (`pcf_csr`).
 *
 * For two PCFs f, g the library computes combination integrals
 *     F(f, g) = r( int_0^inf h(f(t), g(t)) dt )                 (Sec. 2.2)
 * with h(a,b) = |a-b|^p, r(x) = x^(1/p) for the L_p distance (p >= 1) and
 * h(a,b) = a*b, r = id for the L2 inner product, by one linear-time merge walk
 * over the two breakpoint lists per pair (rectangle iteration, Sec. 3 Alg. 1;
 * accumulation, Alg. 2; Eq. simpleint), and assembles them into matrices
 * (Sec. 3.1, "integrated combination matrix").
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller.  The library
 *    allocates nothing and keeps no state between calls; scratch memory is the
 *    caller's `workspace` (size from pcf_workspace_size, 256-byte aligned).
 *    The one exception is pcf_pairwise_noalloc (at the end of this header):
 *    its scratch is a fixed device array inside the library, and it caches
 *    that array's device address per device.
 *  - Work is enqueued on `stream` and returns without synchronizing.  The
 *    return value reports argument errors found on the host.  Problems that
 *    can only be seen in device data (an invalid PCF) are recorded in the
 *    workspace; pcf_check() synchronizes the stream and returns them.  When
 *    the device check fails, the compute kernels of that call skip all work
 *    and the outputs are left unspecified.
 *  - A PCF whose final value differs from that of its partner integrates to
 *    +-inf for that pair (the last rectangle [t_last, inf) adds h * inf when
 *    h != 0 and nothing when h = 0).
 *  - Calls that share a workspace must be ordered on one stream.
 */
#ifndef PCF_H
#define PCF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The CUDA runtime's stream handle type (identical declaration). */
typedef struct CUstream_st* cudaStream_t;

/* Return codes. */
enum pcf_status {
    PCF_OK = 0,
    PCF_EINVAL = 1,    /* bad argument, or invalid PCF data found on the device */
    PCF_ENOWS = 2,     /* workspace missing, misaligned or too small */
    PCF_ECUDA = 3,     /* a CUDA runtime call failed */
    PCF_ETIMEOUT = 4,  /* a bounded device wait gave up */
    PCF_EUNSUPPORTED = 5 /* valid request this build does not implement */
};

/* Element type of times/values/outputs. */
enum pcf_dtype { PCF_F32 = 0, PCF_F64 = 1 };

/* Which combination integral (Sec. 2.2). */
enum pcf_metric {
    PCF_L1 = 0,    /* h = |a-b|,    r = id (root of p = 1)                      */
    PCF_L2 = 1,    /* h = (a-b)^2,  r = sqrt if apply_root                      */
    PCF_LP = 2,    /* h = |a-b|^p,  r = x^(1/p) if apply_root; p >= 1           */
    PCF_GRAM = 3   /* h = a*b,      r = id (L2 inner product / Gram matrix)     */
};

/* Arithmetic of the walk.  Breakpoint comparisons are exact in the input type. */
enum pcf_precision {
    PCF_PREC_F64 = 0,      /* float64 walk and accumulation                     */
    PCF_PREC_F32_COMP = 1, /* float32 walk, every rectangle's term added by Kahan's
                              compensated summation into a (sum, compensation)
                              pair; error <= 2u * sum|terms| + O(n u^2)        */
    PCF_PREC_F32 = 2,      /* float32 walk, plain float32 fused multiply-add    */
    PCF_PREC_F32_BLOCK = 3 /* float32 walk, terms summed by FMA over blocks of at
                              most 16 rectangles, block sums added by Kahan's
                              compensated summation; error <= about
                              18u * sum|terms| (a fraction of the work of
                              PCF_PREC_F32_COMP)                               */
};
/* float64 input walked in a float32 precision keeps every comparison of the
 * walk exact in float64 (Alg. 1 decides which interval ends first, and ties,
 * on the input's times): each interval end gets a 32-bit order key, its rank
 * among the call's interval ends from a device-wide sort of their float64
 * values, and the walk compares keys.  Each rectangle's width is formed from
 * the difference of its ends, each time carried as float32 hi + lo (about 48
 * significant bits), so distinct breakpoints closer than one float32 ulp stay
 * distinct and a width w ending at time t is exact to about u*w + 2^-48*t
 * instead of u*t.  Inputs whose widths must be resolved beyond that (gaps
 * below about 1e-9 relative to their times) need PCF_PREC_F64.  Values are
 * rounded to float32
 * (the walk's arithmetic).  Such a call needs nnz (both collections together
 * for a cross call) below 2^31, else PCF_EUNSUPPORTED.  The p-th root is
 * always taken in float64.
 *
 * PCF_PREC_ROUND_TIMES, or-ed into a float32 precision, asks for the faster
 * packed form instead: float64 times rounded to nearest float32 when packed
 * (8-byte elements; order is kept, times that round together become one
 * breakpoint of both PCFs, and widths carry the rounding of the times, about
 * u * t per breakpoint).  It has no effect on float32 input and is invalid
 * with PCF_PREC_F64.  Every call that shares a prepared workspace
 * (pcf_prepare, PCF_PAIRWISE_PREPARED) must pass the same precision value. */
#define PCF_PREC_ROUND_TIMES 0x100

/* PCF_PREC_AUTO64, or-ed into a float32 precision: walk in that float32
 * precision unless the input's dynamic range asks for float64, decided on
 * the device during validation with no host synchronization (both walks are
 * enqueued; the one not needed returns at once).  A float64 collection needs
 * the float64 walk when a time or value lies outside float32's normal range
 * (above FLT_MAX, or nonzero below FLT_MIN; without this bit such input is
 * rejected, reason 6) or when a gap t_{k+1} - t_k is below 2^-30 t_{k+1} (the
 * float32 walk resolves widths to about 2^-48 t).  The float64 walk's results
 * are those of PCF_PREC_F64.  pcf_walk_promoted reports which walk ran.  The
 * workspace is sized for both forms.  Invalid with PCF_PREC_F64. */
#define PCF_PREC_AUTO64 0x200

/* Output layout of the pairwise matrix. */
enum pcf_layout {
    PCF_OUT_FULL = 0,          /* N x N row-major, both triangles written      */
    PCF_OUT_UPPER_PACKED = 1,  /* row-major upper triangle with the diagonal:
                                  (i, j), i <= j, at i*N - i*(i-1)/2 + (j - i) */
    PCF_OUT_FULL_SORTED = 2    /* N x N row-major in the library's sort order:
                                  entry (s, t) is F(x[perm[s]], x[perm[t]]) with
                                  perm from pcf_sort_order.  The tiles then land
                                  in contiguous blocks instead of being scattered
                                  by the permutation, which keeps the output
                                  writes near the output size in DRAM traffic */
};

/* Workspace purpose for pcf_workspace_size. */
enum pcf_ws_purpose { PCF_WS_FORWARD = 0, PCF_WS_BACKWARD = 1 };

/* pcf_pairwise flags. */
enum pcf_pairwise_flags {
    PCF_PAIRWISE_PREPARED = 1  /* skip validating/packing x: the workspace holds x
                                  as packed by pcf_prepare (or by a previous
                                  pcf_pairwise) with the same x and precision */
};

/* pcf_cross flags. */
enum pcf_cross_flags {
    PCF_CROSS_REUSE_B = 1  /* skip validating/packing B: the workspace still holds
                              B packed by the previous pcf_cross call made with
                              the same B, precision and workspace.  (float64 input
                              in a float32 precision: B's validation and length
                              sort are reused and B is packed again, because its
                              order keys are ranks among A's rows and B) */
};

/* Work decomposition of the walk (pcf_pairwise_ex / pcf_cross_ex).
 *   PCF_SCHED_TILE_1024   32 x 32 pair tiles, one 1024-thread CTA per SM
 *   PCF_SCHED_TILE_512X2  32 x 16 half tiles, two 512-thread CTAs per SM
 *                         (half the shared memory each: smaller windows)
 *   PCF_SCHED_TILE_512X3  32 x 16 half tiles, three 512-thread CTAs per SM
 *                         (at most 40 registers per thread, a third of the
 *                         shared memory each)
 *   PCF_SCHED_MERGEPATH   one warp per pair, the pair's merge split across
 *                         the 32 lanes (for few, long pairs)
 *   PCF_SCHED_AUTO        merge path when there are fewer tiles than half the
 *                         SMs, else TILE_1024 */
enum pcf_sched_kernel {
    PCF_SCHED_AUTO = 0, PCF_SCHED_TILE_1024 = 1, PCF_SCHED_TILE_512X2 = 2,
    PCF_SCHED_MERGEPATH = 3, PCF_SCHED_TILE_512X3 = 4
};

typedef struct pcf_schedule {
    int32_t kernel;       /* enum pcf_sched_kernel */
    int32_t window;       /* tile kernels: elements staged per PCF per window,
                             8 <= window <= the shared-memory maximum; 0 = max */
    int32_t shard_index;  /* multi-GPU split of one call: this call computes
                             only work units u (tiles; pairs for the merge
                             path, in the queue order) with
                             u % shard_count == shard_index and writes only
                             their entries; 0 <= shard_index < shard_count */
    int32_t shard_count;  /* 0 or 1: the whole matrix */
    int32_t reserved[4];  /* must be 0 */
} pcf_schedule;

/* Integration window and weight (pcf_pairwise_ex / pcf_cross_ex).
 * The integrals become int_a^b h(f(t), g(t)) w(t) dt with 0 <= a < b <= inf
 * (Alg. 1 takes the bounds a, b) and w(t) = exp(-lambda t), lambda >= 0,
 * integrated per rectangle through its antiderivative (the time-dependent
 * combinations of Sec. 2.1 and Sec. 3).  For float32 walks a, b and lambda
 * are rounded to float32.  With b < inf nothing diverges.  Tile schedules
 * only (PCF_SCHED_AUTO picks TILE_1024); lambda > 0 runs on TILE_1024. */
typedef struct pcf_window {
    double a;
    double b;
    double lambda;
    int32_t reserved[4];   /* must be 0 */
} pcf_window;

/* A collection of N PCFs in CSR form (device arrays, read only).
 *   offsets[N+1] (int64): PCF i owns entries [offsets[i], offsets[i+1]);
 *                         offsets[0] = 0, offsets[N] = nnz, every PCF n_i >= 1.
 *   times[nnz], values[nnz]: dtype elements; times[offsets[i]] = 0 (or -0),
 *                         strictly increasing within a PCF; all finite. */
typedef struct pcf_csr {
    int64_t n;
    int64_t nnz;
    const int64_t* offsets;
    const void* times;
    const void* values;
    int32_t dtype;      /* enum pcf_dtype */
    int32_t reserved;
} pcf_csr;

/* One requested matrix.  Several may be computed in one walk (fused). */
typedef struct pcf_integral {
    int32_t metric;      /* enum pcf_metric */
    int32_t apply_root;  /* distances: 1 -> F = I^(1/p) (p = 1, 2, p); 0 -> F = I */
    double p;            /* exponent for PCF_LP (>= 1); ignored otherwise */
    void* out;           /* device output, layout and dtype per call */
} pcf_integral;

/* Single-PCF functionals (segment iteration, Sec. 3.2). */
enum pcf_functional {
    PCF_FN_INTEGRAL = 0,   /* h(v) = v:     int_a^b f dt                         */
    PCF_FN_LP = 1          /* h(v) = |v|^p: int_a^b |f|^p dt, root -> the L_p norm */
};

/* Maximum number of pcf_integral entries per call. */
#define PCF_MAX_INTEGRALS 4

/*
 * Bytes of workspace needed for pairwise (y == NULL) or cross (y != NULL) work
 * on these collections at `precision`, for `purpose`.  Host-only; reads only
 * x->n, x->nnz (and y's).  Returns PCF_EINVAL for bad sizes.
 */
int pcf_workspace_size(const pcf_csr* x, const pcf_csr* y, int precision,
                       int purpose, size_t* bytes);

/*
 * Validate, sort by length and pack collection x into the workspace (the
 * first stage of pcf_pairwise), so that several pcf_pairwise calls with
 * PCF_PAIRWISE_PREPARED can reuse it.  Same workspace size as pcf_pairwise.
 */
int pcf_prepare(const pcf_csr* x, int precision, void* workspace, size_t workspace_bytes,
                cudaStream_t stream);

/*
 * Pairwise integrated-combination matrices of one collection (Sec. 3.1).
 * Computes nF <= PCF_MAX_INTEGRALS matrices of x in one pass: validation and
 * packing of x (sorted by length), then one merge walk per unordered pair
 * i <= j whose terms feed every requested integral.
 *   F[k].out: N*N (FULL) or N*(N+1)/2 (UPPER_PACKED) elements of out_dtype.
 *   Distance diagonals are exactly 0; Gram diagonals are ||f_i||^2.
 *   flags: 0 or PCF_PAIRWISE_PREPARED.
 * Returns PCF_OK, PCF_EINVAL (bad enum/argument, p < 1), PCF_ENOWS, PCF_ECUDA.
 */
int pcf_pairwise(const pcf_csr* x, const pcf_integral* F, int nF, int precision,
                 int layout, int out_dtype, int flags, void* workspace,
                 size_t workspace_bytes, cudaStream_t stream);

/*
 * pcf_pairwise with an explicit work decomposition (NULL = PCF_SCHED_AUTO)
 * and integration window (NULL = [0, inf), no weight; see pcf_window).
 * Results are identical for every schedule up to the summation order of the
 * merge-path kernel (which combines 32 partial sums).  An unknown kernel or a
 * window outside its range returns PCF_EINVAL.
 */
int pcf_pairwise_ex(const pcf_csr* x, const pcf_integral* F, int nF, int precision,
                    int layout, int out_dtype, int flags, const pcf_schedule* schedule,
                    const pcf_window* window, void* workspace, size_t workspace_bytes,
                    cudaStream_t stream);

/*
 * FULL pairwise matrices (Sec. 3.1, as pcf_pairwise with PCF_OUT_FULL)
 * streamed to host memory while they are computed.  The walk runs in bands
 * of row blocks of the length-sorted PCFs, shortest first; when a band ends,
 * the rows whose pairs are all written are copied by a copy kernel on
 * copy_stream into host_out, while the next band is computed on stream.
 *   F[k].out:    device N x N matrix of out_dtype (written as by pcf_pairwise).
 *   host_out[k]: host N x N matrix of out_dtype, row-major, page-locked and
 *                device-accessible (cudaHostAlloc, or cudaHostRegister'd);
 *                caller-owned, written by the device until the call's work
 *                on `stream` is complete.
 *   nbands:      0 = 16; 1 = one walk, then one copy.  The first and last
 *                bands are smaller than the others.
 *   schedule:    as pcf_pairwise_ex (NULL = AUTO); no shards.
 *   copy_stream: may equal stream (no overlap).  Work on `stream` enqueued
 *                after this call starts after the last copy.
 * Workspace as pcf_pairwise.  Returns PCF_OK, PCF_EINVAL (as pcf_pairwise,
 * or a host_out pointer the device cannot address), PCF_ENOWS, PCF_ECUDA;
 * data errors are reported by pcf_check.
 */
int pcf_pairwise_to_host(const pcf_csr* x, const pcf_integral* F, int nF, int precision,
                         int out_dtype, const pcf_schedule* schedule, void* const* host_out,
                         int nbands, void* workspace, size_t workspace_bytes,
                         cudaStream_t stream, cudaStream_t copy_stream);

/*
 * Cross matrices between rows [row_begin, row_end) of collection a and all of
 * collection b (the pairwise matrix of Sec. 3.1 taken between two sets).
 * Output k is a (row_end - row_begin) x b->n row-major block with leading
 * dimension ld_out (>= b->n) elements: out[(i - row_begin) * ld_out + j].
 * Block streaming = repeated calls over consecutive row ranges (use
 * PCF_CROSS_REUSE_B after the first).
 */
int pcf_cross(const pcf_csr* a, const pcf_csr* b, int64_t row_begin, int64_t row_end,
              const pcf_integral* F, int nF, int precision, int64_t ld_out,
              int out_dtype, int flags, void* workspace, size_t workspace_bytes,
              cudaStream_t stream);

/* pcf_cross with an explicit work decomposition (NULL = PCF_SCHED_AUTO) and
 * integration window (NULL = [0, inf), no weight). */
int pcf_cross_ex(const pcf_csr* a, const pcf_csr* b, int64_t row_begin, int64_t row_end,
                 const pcf_integral* F, int nF, int precision, int64_t ld_out,
                 int out_dtype, int flags, const pcf_schedule* schedule,
                 const pcf_window* window, void* workspace, size_t workspace_bytes,
                 cudaStream_t stream);

/*
 * Gradient of L = sum_{i,j} G_ij F_ij, F the FULL pairwise matrix of `metric`
 * (p, apply_root as in pcf_pairwise), with respect to x->values and x->times.
 * Not part of the paper (Sec. 3 only remarks that derivatives of a
 * parametrised integrand are available); derived by differentiating each
 * rectangle term of Eq. simpleint.  The walk is recomputed in float64; no
 * forward intermediates are stored.
 *   grad_out: N x N row-major G, dtype grad_dtype.
 *   fwd_out:  N x N row-major F from pcf_pairwise (dtype grad_dtype); needed
 *             only when apply_root = 1 and the exponent is not 1 (the chain
 *             factor r'(I) is taken from F), else may be NULL.
 *   grad_values, grad_times: nnz elements of x->dtype (overwritten).
 * Conventions: d/dt_0 = 0 (t_0 = 0 is fixed).  At a breakpoint both PCFs
 * share, each side's time derivative uses the other PCF's value just before
 * the breakpoint (left derivative).  |a-b| has slope 0 at a = b.  A pair with
 * F_ij = 0 contributes 0 when r'(0) is unbounded.
 * Workspace: pcf_workspace_size(x, NULL, PCF_PREC_F64, PCF_WS_BACKWARD).
 */
int pcf_pairwise_backward(const pcf_csr* x, int metric, double p, int apply_root,
                          const void* fwd_out, const void* grad_out, int grad_dtype,
                          void* grad_values, void* grad_times,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * pcf_pairwise_backward for one GPU's share of a multi-GPU split (NULL
 * schedule = the whole matrix).  Only schedule->shard_index/shard_count are
 * used (kernel must be PCF_SCHED_AUTO or PCF_SCHED_TILE_1024): the call walks
 * the 32 x 32 upper-triangle tiles t (in the order of the forward tile walk)
 * with t % shard_count == shard_index and writes the gradient of the pairs
 * of those tiles (zeros elsewhere).  The shards' outputs sum to the whole
 * gradient (one sum all-reduce, best in float64).
 */
int pcf_pairwise_backward_ex(const pcf_csr* x, int metric, double p, int apply_root,
                             const void* fwd_out, const void* grad_out, int grad_dtype,
                             void* grad_values, void* grad_times, const pcf_schedule* schedule,
                             void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * Pairwise matrices against a non-negative PCF weight w (the weighted L_p
 * distance of Sec. 2.2, the weight multiplying |f - g|^p; the weighted inner
 * product for PCF_GRAM):
 *   F_ij = r( int_0^inf h(x_i(t), x_j(t)) w(t) dt ).
 * w: a collection of exactly one PCF (device arrays, offsets {0, nnz}), with
 * t_0 = 0, increasing finite times and finite values >= 0.  With
 * W(t) = int_0^t w, each rectangle [l, r) of a pair walk adds
 * h * (W(r) - W(l)) (the antiderivative form of Sec. 3): the call moves every
 * breakpoint of x to W(t_k) (float64; intervals where w = 0 vanish; when w's
 * last value is 0 the integrals stop at W(inf)) and computes the unweighted
 * matrices of the moved collection with the precision, layout and schedule
 * given, as pcf_pairwise does.  A pair integrates to +-inf only when its
 * tails differ and w's last value is positive.
 * Workspace: pcf_weighted_workspace_size (caller-owned, 256-byte aligned).
 * Returns as pcf_pairwise; pcf_check reports invalid data of x (reasons
 * 1-6) and of w (reason 10, index = element of w).
 */
int pcf_weighted_workspace_size(const pcf_csr* x, const pcf_csr* w, int precision,
                                size_t* bytes);
int pcf_pairwise_weighted(const pcf_csr* x, const pcf_csr* w, const pcf_integral* F, int nF,
                          int precision, int layout, int out_dtype, const pcf_schedule* schedule,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * Cross matrices against a non-negative PCF weight w: rows [row_begin,
 * row_end) of a against all of b, F_ij = r(int h(a_i, b_j) w dt), output
 * blocks as pcf_cross.  Both collections are moved to W(t) for every call
 * (there is no reuse of b).  Workspace: pcf_cross_weighted_workspace_size.
 */
int pcf_cross_weighted_workspace_size(const pcf_csr* a, const pcf_csr* b, const pcf_csr* w,
                                      int precision, size_t* bytes);
int pcf_cross_weighted(const pcf_csr* a, const pcf_csr* b, int64_t row_begin, int64_t row_end,
                       const pcf_csr* w, const pcf_integral* F, int nF, int precision,
                       int64_t ld_out, int out_dtype, const pcf_schedule* schedule,
                       void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * Single-PCF integrals by segment iteration (Sec. 3.2, Alg. 3):
 *   out[i] = r( int_a^b h(f_i(t)) dt ),  0 <= a < b <= inf,
 * h per pcf_functional; r(x) = x^(1/p) for PCF_FN_LP with apply_root, else x.
 * A PCF whose last value makes h != 0 integrates to +-inf when b = inf.
 * out: x->n elements of out_dtype.  The input is validated as for
 * pcf_pairwise (pcf_check reports invalid data).  Workspace:
 * pcf_workspace_size(x, NULL, PCF_PREC_F64, PCF_WS_FORWARD).  precision:
 * PCF_PREC_F64 (float64 arithmetic) or PCF_PREC_F32_COMP (float32 arithmetic,
 * Kahan-compensated per segment; float64 input rounded to float32).  PCFs of
 * any length: one longer than 30,720 breakpoints is integrated in pieces by
 * several CTAs whose partial sums are added in a fixed order, so repeated
 * calls give the same bits.
 */
int pcf_segment_integrals(const pcf_csr* x, int functional, double p, int apply_root,
                          double a, double b, int precision, void* out, int out_dtype,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * The sort order used by the last pcf_prepare / pcf_pairwise on `workspace`
 * for collection x at `precision`: perm_out[s] (device, x->n int32) = input
 * index of the s-th PCF (ascending length bucket, then time scale for PCFs
 * longer than 256 points; stable).  Stream-ordered copy.
 */
int pcf_sort_order(const pcf_csr* x, int precision, const void* workspace,
                   size_t workspace_bytes, int32_t* perm_out, cudaStream_t stream);

/*
 * Synchronizes `stream` and returns the device-side status recorded in the
 * workspace by the last call: PCF_OK, or PCF_EINVAL with *detail set to the
 * reason code (1 offsets, 2 t_0 != 0, 3 times not increasing, 4 time not
 * finite, 5 value not finite, 6 time or value outside float32 range for a
 * float32 walk, 7 more coincident float32 times than one window holds:
 * only with PCF_PREC_ROUND_TIMES) and
 * *index to the offending entry: an offsets error (reason 1, PCF index) is
 * reported before element errors, and among element errors the smallest
 * element index wins.  Reductions and combinations also report PCF_ENOWS
 * with reason 8 when a result or an intermediate needs more rows than the
 * output capacity or the workspace holds (*index = the rows needed, or the
 * merge positions of the pass that did not fit).  pcf_pairwise_weighted
 * reports an invalid weight with reason 10 (*index = element of the weight).
 * detail/index may be NULL.
 */
int pcf_check(const void* workspace, cudaStream_t stream, int* detail, int64_t* index);

/* ------------------------------------------------------------------------
 * Reductions and combinations of PCFs (Sec. 4; Sec. 2.1)
 * ------------------------------------------------------------------------ */

/* Reductions of a group of m PCFs (Sec. 2.1: reduction operations induced by
 * an associative, symmetric h; the mean and the sample standard deviation). */
enum pcf_reduction {
    PCF_RED_SUM = 0,   /* f_1 + ... + f_m                                        */
    PCF_RED_MEAN = 1,  /* (f_1 + ... + f_m) / m                                  */
    PCF_RED_MAX = 2,   /* pointwise maximum                                      */
    PCF_RED_MIN = 3,   /* pointwise minimum                                      */
    PCF_RED_STD = 4    /* sqrt( sum_i (f_i - mean)^2 / (m - 1) ), m >= 2         */
};

/* Combination functions h of the induced operation h_*(f, g)(t) = h(f(t), g(t)). */
enum pcf_op {
    PCF_OP_ADD = 0, PCF_OP_SUB = 1, PCF_OP_MUL = 2, PCF_OP_MAX = 3, PCF_OP_MIN = 4,
    PCF_OP_SQDIFF = 5  /* (a - b)^2 */
};

/* A caller-owned output collection (device arrays).  Results are float64.
 *   offsets:  [n_out + 1] int64, written by the call (offsets[0] = 0).
 *   times, values: capacity float64 rows each. */
typedef struct pcf_csr_out {
    int64_t capacity;
    int64_t* offsets;
    double* times;
    double* values;
} pcf_csr_out;

/*
 * Result rows: every reduction and combination builds its output with
 * ReducePair (Sec. 4, Alg. 4): the merged breakpoints of its inputs, keeping
 * a breakpoint when t = 0 or when the value changes there (a value equal to
 * the one before is not repeated).  Arithmetic is float64; float32 input is
 * widened exactly.
 */

/*
 * Workspace bytes for pcf_reduce.  PCF_RED_STD also holds the intermediate
 * PCFs (f_i - mean)^2; `std_rows` is the row capacity to reserve for them:
 * 0 = the worst case (m + 1) * x->nnz, or exactly x->nnz + m * (rows of the
 * group means), which pcf_reduce with PCF_RED_MEAN gives.  Ignored for the
 * other reductions.  pcf_reduce uses whatever capacity the workspace it is
 * given holds and checks it on the device (reason 8).
 */
int pcf_reduce_workspace_size(const pcf_csr* x, int64_t group_size, int reduction,
                              int64_t std_rows, size_t* bytes);

/*
 * Reduce each of the x->n / group_size consecutive groups of group_size PCFs
 * to one PCF (x->n must be a multiple of group_size).  The group is reduced
 * by a binary tree of ReducePair nodes (Sec. 4, Fig. 2 with two inputs per
 * node): on each level node k combines items 2k and 2k + 1, and an odd last
 * item moves up unchanged.  MEAN divides the values of the sum by m; STD
 * (m >= 2) reduces the ReducePair results (f_i - mean)^2 by a sum tree and
 * maps v -> sqrt(v / (m - 1)) (the unbiased factor).  After a division or
 * root, a value equal to the one before it is dropped as in Alg. 4.
 * m = 1: SUM, MAX and MIN return the input rows unchanged.
 *   out: group count + 1 offsets; capacity >= x->nnz always suffices.
 * Input validated as for pcf_pairwise.  No host synchronization.
 */
int pcf_reduce(const pcf_csr* x, int64_t group_size, int reduction, pcf_csr_out* out,
               void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* Workspace bytes for pcf_combine(a, b, ...). */
int pcf_combine_workspace_size(const pcf_csr* a, const pcf_csr* b, size_t* bytes);

/*
 * Elementwise combination h_*(a_i, b_i) (ReducePair, Sec. 4, Alg. 4) with
 * h = op, for b->n == a->n, or h_*(a_i, b_0) for every i when b->n == 1.
 *   out: a->n + 1 offsets; capacity >= a->nnz + b->nnz (pairs), or
 *   a->nnz + a->n * b->nnz (one b) always suffices.
 */
int pcf_combine(const pcf_csr* a, const pcf_csr* b, int op, pcf_csr_out* out,
                void* workspace, size_t workspace_bytes, cudaStream_t stream);

/*
 * Work done by the last pcf_reduce / pcf_combine on `workspace` (synchronizes
 * `stream`): *positions = merge positions visited over all its ReducePair
 * passes (one per input breakpoint of every pass), *rows = rows those passes
 * wrote.  With 16-byte (t, v) rows, 16 * (positions + rows) bytes is the
 * least DRAM traffic of the passes.  Either pointer may be NULL.
 */
int pcf_reduce_counters(const void* workspace, cudaStream_t stream, int64_t* positions,
                        int64_t* rows);

/*
 * Self-test of the bounded device waits (no counterpart in the paper).  The
 * reductions turn per-chunk row counts into output positions by decoupled
 * look-back, in which a chunk waits for its predecessors' published counts;
 * every such wait gives up after a bounded number of polls, records reason 9
 * and lets its successors stop.  This call runs that wait for chunk 1 while
 * chunk 0 never publishes, with at most `polls` polls (1 .. 2^20), so the wait
 * runs out: pcf_check(workspace) then returns PCF_ETIMEOUT with reason 9.
 * Workspace: at least 512 bytes, 256-byte aligned.
 */
int pcf_selftest_wait_timeout(int64_t polls, void* workspace, size_t workspace_bytes,
                              cudaStream_t stream);

/* Bytes of the fixed device scratch array behind pcf_pairwise_noalloc. */
#define PCF_NOALLOC_SCRATCH_BYTES (16u << 20)

/*
 * pcf_pairwise without a workspace argument and without any device
 * allocation, for callers that cannot allocate device memory where they
 * need the matrices (an operator interface that only hands over input and
 * output buffers, a service whose device memory budget is fully reserved up
 * front, code that must not call into the allocator after start-up).  The
 * paper has no counterpart; this is an interface convenience.
 *   Same arguments and results as pcf_pairwise with flags = 0, except that
 *   the scratch is a file-scope device array of PCF_NOALLOC_SCRATCH_BYTES
 *   inside the library (held on every GPU that loads the library until the
 *   process exits).  Inputs whose pcf_workspace_size exceeds it return
 *   PCF_ENOWS before any device work.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it; make
 *   that first call before any stream capture.
 *   All calls on a device share the array: each call re-initializes what it
 *   uses, but calls whose GPU work overlaps in time (other streams, other
 *   host threads) race and give wrong results.  Device-side input errors are
 *   recorded in the array and are not reported by this entry point.
 */
int pcf_pairwise_noalloc(const pcf_csr* x, const pcf_integral* F, int nF, int precision,
                         int layout, int out_dtype, cudaStream_t stream);

/*
 * After a call made with PCF_PREC_AUTO64 on `workspace` (pcf_prepare,
 * pcf_pairwise, pcf_pairwise_to_host, pcf_cross): synchronizes `stream` and
 * sets *promoted to 1 when the float64 walk ran (the input's dynamic range
 * asked for it), 0 when the float32 walk did.  PCF_EINVAL for null pointers.
 */
int pcf_walk_promoted(const void* workspace, cudaStream_t stream, int* promoted);

/* Static text for a status code. */
const char* pcf_status_string(int status);

/* Library build identification (static string). */
const char* pcf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PCF_H */
