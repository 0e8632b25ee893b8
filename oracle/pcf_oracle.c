/*
 * pcf_oracle.c -- CPU reference for the PCF integral matrices.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * table or helper with the CUDA library; the product path never calls it.
 *
 * Everything here is plain float64 C, written for readability, not speed:
 *
 *   orc_rectangles      rectangle iteration over [0, inf)     (Sec. 3, Alg. 1)
 *   orc_integral        combine-and-integrate of h(f, g)      (Sec. 3, Alg. 2,
 *                                                              Eq. simpleint)
 *   orc_matrix          pairwise / cross matrices F_ij = r(I_ij)
 *                                                             (Sec. 3.1; Sec. 2.2
 *                                                              for r and h)
 *   orc_integral_ab     Alg. 1/2 over [a, b], optionally with the exponential
 *                       weight w(t) = exp(-lambda t) through its antiderivative
 *                                                             (Sec. 3, Alg. 1
 *                                                              bounds; Sec. 2.1
 *                                                              time-dependent h)
 *   orc_integral_w      int h(f, g) w dt for a non-negative PCF weight w
 *                       (rectangle iteration over three breakpoint lists)
 *                                                             (Sec. 2.2 weighted
 *                                                              L_p; Sec. 2.1
 *                                                              time-dependent h;
 *                                                              Alg. 1/2)
 *   orc_segment_sq      integral of f^2 by segment iteration  (Sec. 3.2, Alg. 3)
 *   orc_segment_integral integral of f or |f|^p over [a, b]    (Sec. 3.2, Alg. 3)
 *   orc_reduce_pair     ReducePair: the PCF h_*(f, g) with repeated values
 *                       dropped                               (Sec. 4, Alg. 4)
 *   orc_reduce          sum / mean / max / min / sample std of groups of PCFs
 *                       by binary reduction trees      (Sec. 4, Fig. 2; mean
 *                                                       and std of Sec. 2.1)
 *   orc_backward        gradient of sum_ij G_ij F_ij with respect to the
 *                       breakpoint values and times (not in the paper; derived
 *                       from Eq. simpleint by differentiating each rectangle)
 *
 * Combination functions h (Sec. 2.2): the L_p distance uses h(a,b) = |a-b|^p
 * with r(x) = x^(1/p); the L2 inner product uses h(a,b) = a*b with r = id.
 *
 * Readings of points the paper leaves open (each one is listed with its reason
 * in the design notes of the repository):
 *  - a PCF is stored as n >= 1 breakpoints t_0 = 0 < t_1 < ... < t_{n-1} with
 *    values v_0..v_{n-1}; v_{n-1} holds on [t_{n-1}, inf).
 *  - the last rectangle [t_last, inf) adds 0 when h(v_f, v_g) = 0 and
 *    h * inf (= +-inf) otherwise (0 * inf is not used).
 *  - |d|^p: p = 1 gives |d|, p = 2 gives d*d, other integer p a left-to-right
 *    product of |d|, non-integer p pow(|d|, p).  The root r uses sqrt for p = 2
 *    and pow(x, 1/p) for other p != 1.
 *  - gradient at a breakpoint that both PCFs share: each side takes the value
 *    of the other PCF just before the breakpoint (left limit), which is what the
 *    simultaneous advance of Alg. 1 hands out.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_L1 = 0, ORC_L2 = 1, ORC_LP = 2, ORC_GRAM = 3 };

/* |d|^p as described in the header comment. */
static double orc_pow_abs(double d, double p)
{
    double a = fabs(d);
    if (p == 1.0) return a;
    if (p == 2.0) return d * d;
    if (p == floor(p) && p > 2.0 && p <= 64.0) {
        double r = a;
        for (int i = 1; i < (int)p; ++i) r = r * a;
        return r;
    }
    return pow(a, p);
}

/* Combination function h of Sec. 2.2 for the requested matrix. */
static double orc_h(int metric, double p, double a, double b)
{
    switch (metric) {
    case ORC_L1: return fabs(a - b);
    case ORC_L2: return (a - b) * (a - b);
    case ORC_LP: return orc_pow_abs(a - b, p);
    default: return a * b;  /* ORC_GRAM */
    }
}

/* Partial derivative of h with respect to its first argument. */
static double orc_dh_da(int metric, double p, double a, double b)
{
    double d = a - b;
    double s = (d > 0.0) ? 1.0 : ((d < 0.0) ? -1.0 : 0.0);
    switch (metric) {
    case ORC_L1: return s;
    case ORC_L2: return 2.0 * d;
    case ORC_LP:
        if (d == 0.0) return 0.0;
        return p * orc_pow_abs(d, p - 1.0) * s;
    default: return b;  /* ORC_GRAM */
    }
}

/* Exponent of the metric (1 for L1, 2 for L2, p for LP, 1 for the Gram). */
static double orc_exponent(int metric, double p)
{
    if (metric == ORC_L1) return 1.0;
    if (metric == ORC_L2) return 2.0;
    if (metric == ORC_LP) return p;
    return 1.0;
}

/* r(x) of Sec. 2.2: x^(1/p) for distances when requested, else x. */
static double orc_root(int metric, double p, int apply_root, double x)
{
    if (!apply_root || metric == ORC_GRAM) return x;
    double e = orc_exponent(metric, p);
    if (e == 1.0) return x;
    if (e == 2.0) return sqrt(x);
    return pow(x, 1.0 / e);
}

/* dr/dx at the integral value x. */
static double orc_droot(int metric, double p, int apply_root, double x)
{
    if (!apply_root || metric == ORC_GRAM) return 1.0;
    double e = orc_exponent(metric, p);
    if (e == 1.0) return 1.0;
    return (1.0 / e) * pow(x, 1.0 / e - 1.0);
}

/*
 * Rectangle iteration of Alg. 1 with a = 0 and b = inf.
 *
 * Two cursors k (into f) and kg (into g) start at the breakpoint at t = 0.
 * Each pass emits the rectangle that starts at the current scanline time
 * with the values f(t), g(t), after moving whichever cursor has the earlier
 * next breakpoint (both on a tie).  When neither can move, the final
 * rectangle reaches to b = inf.  Rectangles are handed to `emit`; the
 * return value is the number of rectangles.
 */
typedef void (*orc_emit_fn)(void* ctx, double l, double r, double vf, double vg,
                            int64_t kf, int64_t kg, int moved_f, int moved_g);

static int64_t orc_walk(const double* tf, const double* vf, int64_t nf,
                        const double* tg, const double* vg, int64_t ng,
                        orc_emit_fn emit, void* ctx)
{
    int64_t k = 0, kg = 0, count = 0;
    double t = 0.0;
    for (;;) {
        double t_prev = t;
        double a = vf[k], b = vg[kg];
        int64_t k_old = k, kg_old = kg;
        int moved_f = 0, moved_g = 0;
        if (k + 1 < nf && kg + 1 < ng) {
            /* sign of delta = t_{k+1} - t'_{k'+1} decides who moves */
            if (tf[k + 1] <= tg[kg + 1]) { k += 1; moved_f = 1; }
            if (tg[kg + 1] <= tf[k_old + 1]) { kg += 1; moved_g = 1; }
        } else if (k + 1 < nf) {
            k += 1; moved_f = 1;
        } else if (kg + 1 < ng) {
            kg += 1; moved_g = 1;
        } else {
            emit(ctx, t_prev, INFINITY, a, b, k_old, kg_old, 0, 0);
            return count + 1;
        }
        t = (tf[k] > tg[kg]) ? tf[k] : tg[kg];
        emit(ctx, t_prev, t, a, b, k_old, kg_old, moved_f, moved_g);
        count += 1;
    }
}

/* ---- rectangles as a list (for tests of Alg. 1 itself) ---- */
typedef struct { double* l; double* r; double* a; double* b; int64_t cap; int64_t n; } orc_rect_list;

static void orc_emit_list(void* ctx, double l, double r, double a, double b,
                          int64_t kf, int64_t kg, int mf, int mg)
{
    (void)kf; (void)kg; (void)mf; (void)mg;
    orc_rect_list* L = (orc_rect_list*)ctx;
    if (L->n < L->cap) {
        L->l[L->n] = l; L->r[L->n] = r; L->a[L->n] = a; L->b[L->n] = b;
    }
    L->n += 1;
}

int64_t orc_rectangles(const double* tf, const double* vf, int64_t nf,
                       const double* tg, const double* vg, int64_t ng,
                       double* l, double* r, double* a, double* b, int64_t cap)
{
    orc_rect_list L = { l, r, a, b, cap, 0 };
    orc_walk(tf, vf, nf, tg, vg, ng, orc_emit_list, &L);
    return L.n;
}

/* ---- Alg. 2: I = sum over rectangles of h(v_f, v_g) * (r - l) ---- */
typedef struct { int metric; double p; double I; } orc_acc;

static void orc_emit_acc(void* ctx, double l, double r, double a, double b,
                         int64_t kf, int64_t kg, int mf, int mg)
{
    (void)kf; (void)kg; (void)mf; (void)mg;
    orc_acc* A = (orc_acc*)ctx;
    double h = orc_h(A->metric, A->p, a, b);
    if (isinf(r)) {
        if (h != 0.0) A->I += h * INFINITY;  /* diverging tail */
        return;
    }
    A->I += h * (r - l);
}

double orc_integral(const double* tf, const double* vf, int64_t nf,
                    const double* tg, const double* vg, int64_t ng,
                    int metric, double p)
{
    orc_acc A = { metric, p, 0.0 };
    orc_walk(tf, vf, nf, tg, vg, ng, orc_emit_acc, &A);
    return A.I;
}

/*
 * Alg. 1 with integration bounds 0 <= a < b <= inf: the cursors start at the
 * last breakpoints <= a, the scanline starts at a, and every rectangle's right
 * end is clipped to b; the walk stops once the scanline reaches b.
 * Accumulation of Alg. 2, or -- for the time-dependent combination
 * h(x, y, t) = h(x, y) w(t) with w(t) = exp(-lambda t) -- the antiderivative
 * form of Sec. 3: each rectangle adds H(v_f, v_g, r) - H(v_f, v_g, l) with
 * H(x, y, t) = h(x, y) W(t), W(t) = -exp(-lambda t) / lambda.  The difference
 * W(r) - W(l) is evaluated as exp(-lambda l) * (-expm1(-lambda (r - l))) /
 * lambda, the same quantity without the cancellation of two close
 * exponentials; lambda = 0 is the unweighted case.
 */
double orc_integral_ab(const double* tf, const double* vf, int64_t nf,
                       const double* tg, const double* vg, int64_t ng,
                       int metric, double p, double a, double b, double lambda)
{
    int64_t k = 0, kg = 0;
    while (k + 1 < nf && tf[k + 1] <= a) k++;
    while (kg + 1 < ng && tg[kg + 1] <= a) kg++;
    double t = a, I = 0.0;
    while (t < b) {
        double t_prev = t;
        double h = orc_h(metric, p, vf[k], vg[kg]);
        int64_t k_old = k;
        if (k + 1 < nf && kg + 1 < ng) {
            if (tf[k + 1] <= tg[kg + 1]) k += 1;
            if (tg[kg + 1] <= tf[k_old + 1]) kg += 1;
        } else if (k + 1 < nf) {
            k += 1;
        } else if (kg + 1 < ng) {
            kg += 1;
        } else {
            t = b;                            /* last rectangle reaches b */
            if (isinf(b) && lambda == 0.0) {  /* unweighted tail [t, inf) */
                if (h != 0.0) I += h * INFINITY;
                return I;
            }
            /* weighted: exp(-lambda t_prev) / lambda for b = inf, finite */
        }
        if (t < b) {
            double nt = (tf[k] > tg[kg]) ? tf[k] : tg[kg];
            t = nt < b ? nt : b;
        }
        double dw;
        if (lambda == 0.0) dw = t - t_prev;
        else dw = exp(-lambda * t_prev) * (-expm1(-lambda * (t - t_prev))) / lambda;
        I += h * dw;
    }
    return I;
}

/*
 * Weighted combination integral int_0^inf h(f(t), g(t)) w(t) dt for a
 * non-negative PCF weight w (the weighted L_p distance of Sec. 2.2 with the
 * weight multiplying |f - g|^p, and the weighted inner product), by rectangle
 * iteration over the three breakpoint lists T_f, T_g, T_w: the scanline moves
 * to the earliest next breakpoint of the three, every list whose next
 * breakpoint is there moves with it, and each rectangle [l, r) on which f, g
 * and w are constant adds h(f, g) * w * (r - l).  The last rectangle,
 * [t_last, inf), adds 0 when h * w = 0 there and +-inf otherwise.
 */
double orc_integral_w(const double* tf, const double* vf, int64_t nf,
                      const double* tg, const double* vg, int64_t ng,
                      const double* tw, const double* vw, int64_t nw,
                      int metric, double p)
{
    int64_t i = 0, j = 0, k = 0;
    double t = 0.0, I = 0.0;
    for (;;) {
        double next = INFINITY;
        if (i + 1 < nf && tf[i + 1] < next) next = tf[i + 1];
        if (j + 1 < ng && tg[j + 1] < next) next = tg[j + 1];
        if (k + 1 < nw && tw[k + 1] < next) next = tw[k + 1];
        const double hw = orc_h(metric, p, vf[i], vg[j]) * vw[k];
        if (isinf(next)) {
            if (hw != 0.0) I += hw * INFINITY;
            return I;
        }
        I += hw * (next - t);
        t = next;
        if (i + 1 < nf && tf[i + 1] == next) i += 1;
        if (j + 1 < ng && tg[j + 1] == next) j += 1;
        if (k + 1 < nw && tw[k + 1] == next) k += 1;
    }
}

/* Number of rectangles of the pair = |T_f u T_g| (the merge-step count). */
int64_t orc_merge_steps(const double* tf, int64_t nf, const double* tg, int64_t ng)
{
    int64_t i = 0, j = 0, m = 0;
    while (i < nf || j < ng) {
        if (j >= ng || (i < nf && tf[i] < tg[j])) { i++; }
        else if (i >= nf || tg[j] < tf[i]) { j++; }
        else { i++; j++; }
        m++;
    }
    return m;
}

/* ---- matrices ---- */
typedef struct {
    int64_t na, nb;
    const int64_t *oa, *ob;
    const double *ta, *va, *tb, *vb;
    int metric; double p; int apply_root;
    int symmetric;       /* pairwise: fill only j >= i and mirror */
    double* out;         /* na x nb row-major */
    int64_t next_row;
    pthread_mutex_t lock;
} orc_job;

static void orc_do_row(orc_job* J, int64_t i)
{
    const double* tf = J->ta + J->oa[i];
    const double* vf = J->va + J->oa[i];
    int64_t nf = J->oa[i + 1] - J->oa[i];
    int64_t j0 = J->symmetric ? i : 0;
    for (int64_t j = j0; j < J->nb; ++j) {
        const double* tg = J->tb + J->ob[j];
        const double* vg = J->vb + J->ob[j];
        int64_t ng = J->ob[j + 1] - J->ob[j];
        double I = orc_integral(tf, vf, nf, tg, vg, ng, J->metric, J->p);
        double F = orc_root(J->metric, J->p, J->apply_root, I);
        J->out[i * J->nb + j] = F;
        if (J->symmetric) J->out[j * J->nb + i] = F;
    }
}

static void* orc_worker(void* arg)
{
    orc_job* J = (orc_job*)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t i = J->next_row++;
        pthread_mutex_unlock(&J->lock);
        if (i >= J->na) return NULL;
        orc_do_row(J, i);
    }
}

/*
 * F(C) of Sec. 3.1.  With (ob, tb, vb) == NULL the matrix is the pairwise
 * matrix of set A (symmetric; rows [row_begin, row_end) of it); otherwise the
 * cross matrix rows of A x B.  `out` is (row_end - row_begin) x nb.
 */
void orc_matrix(int64_t na, const int64_t* oa, const double* ta, const double* va,
                int64_t nb, const int64_t* ob, const double* tb, const double* vb,
                int64_t row_begin, int64_t row_end,
                int metric, double p, int apply_root, double* out, int nthreads)
{
    orc_job J;
    memset(&J, 0, sizeof J);
    int pairwise = (ob == NULL);
    /* rows of A restricted to [row_begin, row_end) */
    J.na = row_end - row_begin;
    J.oa = oa + row_begin;
    J.ta = ta; J.va = va;
    J.nb = pairwise ? na : nb;
    J.ob = pairwise ? oa : ob;
    J.tb = pairwise ? ta : tb;
    J.vb = pairwise ? va : vb;
    J.metric = metric; J.p = p; J.apply_root = apply_root;
    J.symmetric = pairwise && row_begin == 0 && row_end == na;
    J.out = out;
    J.next_row = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads == 1) {
        orc_worker(&J);
    } else {
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, orc_worker, &J);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        free(th);
    }
    pthread_mutex_destroy(&J.lock);
    (void)J;
    /* row_begin > 0 reuses the same loop: indices of oa are shifted above, and
     * for the pairwise case the columns still run over all of A. */
}

/*
 * Alg. 3 (segment iteration) over [a, b]: start at the segment containing a,
 * emit segments [l, r) clipped to [a, b], each contributing h(v) (r - l), stop
 * at b.  kind 0: h(v) = v (the integral of f); kind 1: h(v) = |v|^p.  A last
 * segment reaching b = inf adds 0 when h = 0 and h * inf otherwise.
 */
double orc_segment_integral(const double* t, const double* v, int64_t n, int kind, double p,
                            double a, double b)
{
    int64_t k = 0;
    while (k + 1 < n && t[k + 1] <= a) k++;          /* k = max{i : t_i <= a} */
    double l = a, I = 0.0;
    for (;;) {
        double h = (kind == 0) ? v[k] : orc_pow_abs(v[k], p);
        double r = (k + 1 < n) ? t[k + 1] : INFINITY;
        if (r >= b) r = b;
        if (isinf(r)) {
            if (h != 0.0) I += h * INFINITY;
            return I;
        }
        I += h * (r - l);
        if (r >= b) return I;
        l = r;
        k++;
    }
}

/* Alg. 3 (segment iteration) for the integral of f^2 over [0, inf). */
double orc_segment_sq(const double* t, const double* v, int64_t n)
{
    double I = 0.0;
    for (int64_t k = 0; k + 1 < n; ++k) I += v[k] * v[k] * (t[k + 1] - t[k]);
    if (v[n - 1] != 0.0) I += v[n - 1] * v[n - 1] * INFINITY;
    return I;
}

/* ---- adjoint ---- */
typedef struct {
    int metric; double p; double w;
    double *gvf, *gtf, *gvg, *gtg;   /* gradient slices of f and g */
    const double *vf_arr, *vg_arr;
} orc_grad_ctx;

/*
 * d/dv of a rectangle [l, r) with values (a, b): w * dh/da * (r - l) for the
 * f side and w * dh/db * (r - l) = w * dh/da(b, a) * (r - l) for the g side
 * (h is symmetric).  When the scanline moves f past its breakpoint t_{k+1}
 * (the end of this rectangle), d/dt_{k+1} gains w * (h(v_k, b) - h(v_{k+1}, b))
 * with b the value of g just before the breakpoint; likewise for g.
 */
static void orc_emit_grad(void* ctx, double l, double r, double a, double b,
                          int64_t kf, int64_t kg, int mf, int mg)
{
    orc_grad_ctx* C = (orc_grad_ctx*)ctx;
    double da = orc_dh_da(C->metric, C->p, a, b);
    double db = orc_dh_da(C->metric, C->p, b, a);
    if (isinf(r)) {
        if (da != 0.0) C->gvf[kf] += C->w * da * INFINITY;
        if (db != 0.0) C->gvg[kg] += C->w * db * INFINITY;
        return;
    }
    C->gvf[kf] += C->w * da * (r - l);
    C->gvg[kg] += C->w * db * (r - l);
    if (mf) {
        double a_new = C->vf_arr[kf + 1];
        C->gtf[kf + 1] += C->w * (orc_h(C->metric, C->p, a, b) -
                                  orc_h(C->metric, C->p, a_new, b));
    }
    if (mg) {
        double b_new = C->vg_arr[kg + 1];
        C->gtg[kg + 1] += C->w * (orc_h(C->metric, C->p, b, a) -
                                  orc_h(C->metric, C->p, b_new, a));
    }
}

/*
 * Gradient of L = sum_{i,j} G_ij F_ij (G is n x n row-major, F the pairwise
 * matrix of `metric`) with respect to values[nnz] and times[nnz].  Pairs with
 * i != j are walked once with weight (G_ij + G_ji) r'(I_ij); a pair whose
 * integral is 0 while r' is unbounded there contributes 0.  The Gram diagonal
 * F_ii = int f_i^2 is differentiated by segment iteration (both arguments of
 * h move together); distance diagonals are identically 0.
 */
void orc_backward(int64_t n, const int64_t* off, const double* t, const double* v,
                  int metric, double p, int apply_root, const double* G,
                  double* grad_v, double* grad_t)
{
    int64_t nnz = off[n];
    memset(grad_v, 0, sizeof(double) * (size_t)nnz);
    memset(grad_t, 0, sizeof(double) * (size_t)nnz);
    for (int64_t i = 0; i < n; ++i) {
        const double* ti = t + off[i];
        const double* vi = v + off[i];
        int64_t ni = off[i + 1] - off[i];
        for (int64_t j = i + 1; j < n; ++j) {
            const double* tj = t + off[j];
            const double* vj = v + off[j];
            int64_t nj = off[j + 1] - off[j];
            double gsum = G[i * n + j] + G[j * n + i];
            double w = gsum;
            if (apply_root && metric != ORC_GRAM && orc_exponent(metric, p) != 1.0) {
                double I = orc_integral(ti, vi, ni, tj, vj, nj, metric, p);
                if (I == 0.0) continue;
                w = gsum * orc_droot(metric, p, apply_root, I);
            }
            orc_grad_ctx C = { metric, p, w, grad_v + off[i], grad_t + off[i],
                               grad_v + off[j], grad_t + off[j], vi, vj };
            orc_walk(ti, vi, ni, tj, vj, nj, orc_emit_grad, &C);
        }
        if (metric == ORC_GRAM) {
            double w = G[i * n + i];
            double* gv = grad_v + off[i];
            double* gt = grad_t + off[i];
            for (int64_t k = 0; k < ni; ++k) {
                double len = (k + 1 < ni) ? (ti[k + 1] - ti[k]) : INFINITY;
                if (isinf(len)) {
                    if (vi[k] != 0.0) gv[k] += w * 2.0 * vi[k] * INFINITY;
                } else {
                    gv[k] += w * 2.0 * vi[k] * len;
                }
                if (k >= 1) gt[k] += w * (vi[k - 1] * vi[k - 1] - vi[k] * vi[k]);
            }
        }
    }
}

/* ===================================================================== */
/* Reductions (Sec. 4): ReducePair (Alg. 4) and binary reduction trees.   */
/* ===================================================================== */

/* Combination functions h of the induced operations h_* (Sec. 2.1). */
enum { ORC_OP_ADD = 0, ORC_OP_SUB = 1, ORC_OP_MUL = 2, ORC_OP_MAX = 3, ORC_OP_MIN = 4,
       ORC_OP_SQDIFF = 5 };

static double orc_op(int op, double a, double b)
{
    switch (op) {
    case ORC_OP_ADD: return a + b;
    case ORC_OP_SUB: return a - b;
    case ORC_OP_MUL: return a * b;
    case ORC_OP_MAX: return a >= b ? a : b;
    case ORC_OP_MIN: return a <= b ? a : b;
    default: { double d = a - b; return d * d; }   /* ORC_OP_SQDIFF */
    }
}

/*
 * Alg. 4 (ReducePair): walk the rectangles of f and g (Alg. 1); for each
 * rectangle R compute v = h(R.v_f, R.v_g) and append the breakpoint (R.l, v)
 * when R.l = 0 or v differs from the previous rectangle's v.  The output
 * holds at most nf + ng rows; the row count is returned.
 */
typedef struct { int op; double* t; double* v; int64_t n; double v_last; } orc_rp;

static void orc_emit_rp(void* ctx, double l, double r, double a, double b,
                        int64_t kf, int64_t kg, int mf, int mg)
{
    (void)r; (void)kf; (void)kg; (void)mf; (void)mg;
    orc_rp* R = (orc_rp*)ctx;
    double v = orc_op(R->op, a, b);
    if (l == 0.0 || v != R->v_last) {
        R->t[R->n] = l;
        R->v[R->n] = v;
        R->n += 1;
    }
    R->v_last = v;
}

int64_t orc_reduce_pair(const double* tf, const double* vf, int64_t nf,
                        const double* tg, const double* vg, int64_t ng, int op,
                        double* out_t, double* out_v)
{
    orc_rp R = { op, out_t, out_v, 0, 0.0 };
    orc_walk(tf, vf, nf, tg, vg, ng, orc_emit_rp, &R);
    return R.n;
}

/* A PCF owned by the tree code. */
typedef struct { double* t; double* v; int64_t n; } orc_pcf;

/* A copy of an input PCF.  A breakpoint at -0.0 (accepted as t_0 = 0) is
 * stored as +0.0, the t_0 that ReducePair's first rectangle carries. */
static orc_pcf orc_pcf_copy(const double* t, const double* v, int64_t n)
{
    orc_pcf p;
    p.t = (double*)malloc(sizeof(double) * (size_t)n);
    p.v = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t k = 0; k < n; ++k) p.t[k] = (t[k] == 0.0) ? 0.0 : t[k];
    memcpy(p.v, v, sizeof(double) * (size_t)n);
    p.n = n;
    return p;
}

static void orc_pcf_free(orc_pcf* p)
{
    free(p->t);
    free(p->v);
    p->t = p->v = NULL;
    p->n = 0;
}

static orc_pcf orc_pcf_pair(const orc_pcf* f, const orc_pcf* g, int op)
{
    orc_pcf p;
    p.t = (double*)malloc(sizeof(double) * (size_t)(f->n + g->n));
    p.v = (double*)malloc(sizeof(double) * (size_t)(f->n + g->n));
    p.n = orc_reduce_pair(f->t, f->v, f->n, g->t, g->v, g->n, op, p.t, p.v);
    return p;
}

/*
 * Binary reduction tree (Fig. 2 with two inputs per node): level by level,
 * item k of the next level is ReducePair(item 2k, item 2k + 1); an odd last
 * item moves up unchanged (the No-Op node of Fig. 2).  Consumes `items`
 * (m >= 1) and returns the root.
 */
static orc_pcf orc_tree(orc_pcf* items, int64_t m, int op)
{
    while (m > 1) {
        int64_t half = m / 2;
        for (int64_t k = 0; k < half; ++k) {
            orc_pcf r = orc_pcf_pair(&items[2 * k], &items[2 * k + 1], op);
            orc_pcf_free(&items[2 * k]);
            orc_pcf_free(&items[2 * k + 1]);
            items[k] = r;
        }
        if (m % 2) {
            items[half] = items[m - 1];
            m = half + 1;
        } else {
            m = half;
        }
    }
    return items[0];
}

/* Values mapped by v -> v / s (kind 0) or sqrt(v / s) (kind 1); a breakpoint
 * is kept when t = 0 or its mapped value differs from the previous one. */
static orc_pcf orc_map(const orc_pcf* f, int kind, double s)
{
    orc_pcf p;
    p.t = (double*)malloc(sizeof(double) * (size_t)f->n);
    p.v = (double*)malloc(sizeof(double) * (size_t)f->n);
    p.n = 0;
    double last = 0.0;
    for (int64_t k = 0; k < f->n; ++k) {
        double w = f->v[k] / s;
        if (kind == 1) w = sqrt(w);
        if (k == 0 || w != last) {
            p.t[p.n] = f->t[k];
            p.v[p.n] = w;
            p.n += 1;
        }
        last = w;
    }
    return p;
}

enum { ORC_RED_SUM = 0, ORC_RED_MEAN = 1, ORC_RED_MAX = 2, ORC_RED_MIN = 3, ORC_RED_STD = 4 };

/*
 * One group of m PCFs (rows [0, m) of off/t/v) reduced to one PCF:
 *   SUM, MAX, MIN: the tree with h = a + b, max, min;
 *   MEAN: (1/m) times the SUM tree (Sec. 2.1), the factor applied as v / m;
 *   STD:  the sample standard deviation of Sec. 2.1,
 *         sqrt( (1/(m-1)) sum_i (f_i - mean)^2 ), each (f_i - mean)^2 a
 *         ReducePair with h = (a - b)^2, summed by the SUM tree (m >= 2).
 */
static orc_pcf orc_reduce_one(int64_t m, const int64_t* off, const double* t, const double* v,
                              int red)
{
    orc_pcf* items = (orc_pcf*)malloc(sizeof(orc_pcf) * (size_t)m);
    for (int64_t i = 0; i < m; ++i)
        items[i] = orc_pcf_copy(t + off[i], v + off[i], off[i + 1] - off[i]);
    int op = red == ORC_RED_MAX ? ORC_OP_MAX : red == ORC_RED_MIN ? ORC_OP_MIN : ORC_OP_ADD;
    orc_pcf root = orc_tree(items, m, op);
    if (red == ORC_RED_SUM || red == ORC_RED_MAX || red == ORC_RED_MIN) {
        free(items);
        return root;
    }
    orc_pcf mean = orc_map(&root, 0, (double)m);
    orc_pcf_free(&root);
    if (red == ORC_RED_MEAN) {
        free(items);
        return mean;
    }
    for (int64_t i = 0; i < m; ++i) {
        orc_pcf fi = { (double*)(t + off[i]), (double*)(v + off[i]), off[i + 1] - off[i] };
        items[i] = orc_pcf_pair(&fi, &mean, ORC_OP_SQDIFF);
    }
    orc_pcf ss = orc_tree(items, m, ORC_OP_ADD);
    orc_pcf sd = orc_map(&ss, 1, (double)(m - 1));
    orc_pcf_free(&ss);
    orc_pcf_free(&mean);
    free(items);
    return sd;
}

typedef struct {
    int64_t groups, m;
    const int64_t* off; const double* t; const double* v;
    int red;
    orc_pcf* out;
    int64_t next;
    pthread_mutex_t lock;
} orc_red_job;

static void* orc_red_worker(void* arg)
{
    orc_red_job* J = (orc_red_job*)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t g = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (g >= J->groups) return NULL;
        J->out[g] = orc_reduce_one(J->m, J->off + g * J->m, J->t, J->v, J->red);
    }
}

/*
 * Reduce each of `groups` consecutive groups of m PCFs (CSR off/t/v with
 * groups * m rows) to one PCF.  Results go to out_off[groups + 1],
 * out_t/out_v (capacity `cap` rows); returns the total row count, or -1 when
 * `cap` is too small (out_off is then filled with the needed offsets).
 */
int64_t orc_reduce(int64_t groups, int64_t m, const int64_t* off, const double* t,
                   const double* v, int red, int64_t* out_off, double* out_t, double* out_v,
                   int64_t cap, int nthreads)
{
    orc_red_job J;
    memset(&J, 0, sizeof J);
    J.groups = groups; J.m = m; J.off = off; J.t = t; J.v = v; J.red = red;
    J.out = (orc_pcf*)calloc((size_t)(groups > 0 ? groups : 1), sizeof(orc_pcf));
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads == 1 || groups < 2) {
        orc_red_worker(&J);
    } else {
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, orc_red_worker, &J);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        free(th);
    }
    pthread_mutex_destroy(&J.lock);
    int64_t total = 0;
    out_off[0] = 0;
    for (int64_t g = 0; g < groups; ++g) {
        total += J.out[g].n;
        out_off[g + 1] = total;
    }
    int64_t rc = total <= cap ? total : -1;
    if (rc >= 0)
        for (int64_t g = 0; g < groups; ++g) {
            memcpy(out_t + out_off[g], J.out[g].t, sizeof(double) * (size_t)J.out[g].n);
            memcpy(out_v + out_off[g], J.out[g].v, sizeof(double) * (size_t)J.out[g].n);
        }
    for (int64_t g = 0; g < groups; ++g) orc_pcf_free(&J.out[g]);
    free(J.out);
    return rc;
}
