/*
 * CPU oracle for the first-order upwind Eikonal solver of Henriksen, You and
 * Pingali, "Exploiting Asynchronous Priority Scheduling in Parallel Eikonal
 * Solvers" (arXiv 2103.05694).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * definition that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library's product path never does.  It shares no code, header or constant
 * with the CUDA sources.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -std=c11 -fPIC -shared.
 * Contraction of a*b+c into a fused multiply-add is forbidden: every float
 * operation below is a separately rounded IEEE-754 binary64 operation
 * (round to nearest even), exactly as written.
 *
 * Notation follows the paper.  A grid is 2D or 3D, C-order, x contiguous.
 * Axis k = 0 is x (stride 1), k = 1 is y, k = 2 is z.  For a non-source cell
 * n, a_k is the smaller arrival time of its two neighbours along axis k
 * (t_H and t_V of the Background section); an off-grid neighbour counts as
 * +inf.
 *
 * The update form is the paper's exactly monotone rounding d-bar
 * ("Achieving Exact Monotonicity with Finite Precision Arithmetic"):
 *   r = fl(h / v_n),  c = fl(r * r),
 *   G(tau) = fl(...fl(fl(q_0 + q_1) + q_2)),  q_k = fl(m_k * m_k),
 *   m_k = max(fl(tau - a_k), 0),
 *   d-bar = the smallest double tau with G(tau) >= c  (+inf if every a_k is +inf).
 * The max(., 0) terms are the max{D^-, -D^+, 0} of the differencing scheme
 * (Eq. finite_difference), so one definition covers the one-sided case of
 * Algorithm 1 and the quadratic case of Eq. difference_as_root.  In the
 * quadratic regime fl(fl(A + B) - c) >= 0 holds exactly when fl(A + B) >= c,
 * so this equals the paper's "alpha is nonnegative" condition.  The right
 * hand side is read as (h/v)^2 (the printed h^2/v is a typo: Tables 1 and 2
 * reproduce only with (h/v)^2, and Table 2 only with c = fl(fl(h/v)^2)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF (1.0 / 0.0)

/* ---------------------------------------------------------------------------
 * Scalar forms of the local update (section "Loss of Monotonicity With
 * Floating Point Arithmetic" and "Mitigation Strategies").
 * ------------------------------------------------------------------------- */

/* d-tilde: the classical explicit root (Loss of Monotonicity section, the
 * formula right before Table 1), with the right-hand side (h/v)^2. */
double orc_dtilde(double v, double h, double tH, double tV)
{
    double r = h / v;
    double c = r * r;
    double s = tH + tV;
    double q = tH * tH + tV * tV;
    double disc = s * s - 2.0 * (q - c);
    return 0.5 * (s + sqrt(disc));
}

/* d-hat: the rearranged explicit root (Mitigation Strategies, the formula
 * before Table 2).  c = fl(fl(h/v)^2) is what reproduces Table 2. */
double orc_dhat(double v, double h, double tH, double tV)
{
    double r = h / v;
    double c = r * r;
    double d = tH - tV;
    double disc = 2.0 * c - d * d;
    return 0.5 * (tH + tV + sqrt(disc));
}

/* d-hat followed by Newton's method on alpha(tau) = (tau - tH)^2 + (tau - tV)^2
 * - c = 0: the variant the Achieving Exact Monotonicity section reports as
 * deterministic in its tests although it does not follow d-bar's rounding
 * semantics.  The paper gives no stopping rule.  This reading stops when an
 * iterate repeats the previous one, when the derivative 2 (mH + mV) is not
 * positive, or after ORC_NEWTON_ITERS steps. */
#define ORC_NEWTON_ITERS 4
double orc_newton(double v, double h, double tH, double tV)
{
    double r = h / v;
    double c = r * r;
    double tau = orc_dhat(v, h, tH, tV);
    for (int k = 0; k < ORC_NEWTON_ITERS; ++k) {
        double mH = tau - tH;
        double mV = tau - tV;
        double alpha = (mH * mH + mV * mV) - c;
        double slope = 2.0 * (mH + mV);
        if (!(slope > 0.0)) break;
        double next = tau - alpha / slope;
        if (next == tau) break;
        tau = next;
    }
    return tau;
}

/* Per-cell constant of the update: c = fl(fl(h/v)^2) (Eq. difference_as_root
 * with the (h/v)^2 reading; Table 2 pins the two roundings). */
double orc_cell_c(double v, double h)
{
    double r = h / v;
    return r * r;
}

/* G(tau): the monotone root function (alpha plus c) over the active axes,
 * terms summed in axis order x, y, z. */
double orc_G(double tau, const double *a, int D)
{
    double g = 0.0;
    for (int k = 0; k < D; ++k) {
        double m = tau - a[k];
        if (!(m > 0.0)) m = 0.0;     /* max(., 0); a_k = +inf gives -inf -> 0 */
        g = g + m * m;
    }
    return g;
}

static double orc_min_of(const double *a, int D)
{
    double m = ORC_INF;
    for (int k = 0; k < D; ++k) if (a[k] < m) m = a[k];
    return m;
}

static double next_up(double x) { return nextafter(x, ORC_INF); }
static double next_down(double x) { return nextafter(x, -ORC_INF); }

/* The starting guess for d-bar, in the paper's order: Algorithm 1's case
 * split between the one-sided update min + h/v and the quadratic root, the
 * quadratic root taken in the rearranged form d-hat; the 3D case adds the
 * third axis the same way.  Only a guess: the exact answer is fixed below. */
static double orc_dbar_guess(const double *a_in, int D, double r, double c)
{
    double b[3];
    int n = 0;
    for (int k = 0; k < D; ++k) if (a_in[k] < ORC_INF) b[n++] = a_in[k];
    /* sort the finite minima ascending (n <= 3) */
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (b[j] < b[i]) { double s = b[i]; b[i] = b[j]; b[j] = s; }
    double g = b[0] + r;                          /* one-sided update */
    if (n >= 2 && fabs(b[1] - b[0]) < r) {        /* quadratic case */
        double d = b[1] - b[0];
        g = 0.5 * (b[0] + b[1] + sqrt(2.0 * c - d * d));
        if (n == 3 && g > b[2]) {                  /* all three axes upwind */
            double u1 = b[1] - b[0], u2 = b[2] - b[0];
            double s = u1 + u2;
            double disc = s * s - 3.0 * (u1 * u1 + u2 * u2 - c);
            if (disc >= 0.0) g = b[0] + (s + sqrt(disc)) / 3.0;
        }
    }
    if (!(g >= b[0])) g = b[0];
    return g;
}

/* d-bar by the "standard techniques" the paper mentions: start from the
 * explicit guess and step one ulp at a time until tau is the smallest double
 * with G(tau) >= c.  G is non-decreasing in tau, so the set
 * {tau : G(tau) >= c} is an interval [d-bar, +inf] and both loops end. */
double orc_dbar(const double *a, int D, double r, double c)
{
    double amin = orc_min_of(a, D);
    if (amin == ORC_INF) return ORC_INF;
    double g = orc_dbar_guess(a, D, r, c);
    while (orc_G(g, a, D) < c) g = next_up(g);
    while (g > amin && orc_G(next_down(g), a, D) >= c) g = next_down(g);
    return g;
}

static uint64_t dbits(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static double bitsd(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }

/* d-bar a second, independent way: bisection over the bit patterns of the
 * non-negative doubles, whose integer order is their numeric order.
 * G(a_min) = 0 < c and G(a_min + 2 sqrt(c)) >= 4c(1 - eps) >= c. */
double orc_dbar_bisect(const double *a, int D, double c)
{
    double amin = orc_min_of(a, D);
    if (amin == ORC_INF) return ORC_INF;
    uint64_t lo = dbits(amin);
    uint64_t hi = dbits(amin + 2.0 * sqrt(c));
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (orc_G(bitsd(mid), a, D) >= c) hi = mid; else lo = mid;
    }
    return bitsd(hi);
}

/* One application of Algorithm 1 (the Eikonal update operator) with an
 * explicit root in place of Eq. difference_as_root, for the ablation of the
 * Mitigation Strategies section (2D): form 1 = d-tilde (the classical root, "no
 * mitigation"), form 2 = d-hat (the rearranged root), form 3 = d-hat then
 * Newton's method (orc_newton).  One-sided when |tH - tV| >= h/v or one minimum
 * is +inf: min(tH, tV) + h/v.  form 0 = d-bar.  +inf when both minima are +inf. */
double orc_update_form(int form, double v, double h, double tH, double tV)
{
    double r = h / v;
    if (form == 0) {
        double a[2] = {tH, tV};
        return orc_dbar(a, 2, r, r * r);
    }
    double lo = tH < tV ? tH : tV;
    if (lo == ORC_INF) return ORC_INF;
    if (tH == ORC_INF || tV == ORC_INF) return lo + r;
    double d = tH - tV;
    if (fabs(d) >= r) return lo + r;
    if (form == 1) return orc_dtilde(v, h, tH, tV);
    if (form == 2) return orc_dhat(v, h, tH, tV);
    return orc_newton(v, h, tH, tV);
}

/* ---------------------------------------------------------------------------
 * Grid helpers.
 * ------------------------------------------------------------------------- */

typedef struct {
    int D;                 /* 2 or 3 */
    int64_t n[3];          /* extent per axis k (x, y, z) */
    int64_t s[3];          /* stride per axis k */
    int64_t N;             /* number of cells */
} orc_grid;

/* dims are C-order (slowest first): {ny, nx} or {nz, ny, nx}. */
static int orc_grid_make(orc_grid *g, int ndim, const int64_t *dims)
{
    if (ndim < 1 || ndim > 3) return -1;
    g->D = ndim;
    int64_t stride = 1;
    for (int k = 0; k < ndim; ++k) {
        g->n[k] = dims[ndim - 1 - k];
        g->s[k] = stride;
        if (g->n[k] < 1) return -1;
        stride *= g->n[k];
    }
    g->N = stride;
    return 0;
}

/* a_k for cell idx: min of the two neighbours along axis k, +inf off-grid
 * (t_H, t_V in the Background section; Algorithm 1). */
static void orc_axis_minima(const orc_grid *g, const double *t, int64_t idx, double *a)
{
    int64_t rem = idx;
    for (int k = 0; k < g->D; ++k) {
        int64_t coord = rem % g->n[k];
        rem /= g->n[k];
        double lo = (coord > 0) ? t[idx - g->s[k]] : ORC_INF;
        double hi = (coord + 1 < g->n[k]) ? t[idx + g->s[k]] : ORC_INF;
        a[k] = lo < hi ? lo : hi;
    }
}

/* UpdateNode (Algorithm 1) with the d-bar rounding: the value the operator
 * computes at a non-source cell from the current field. */
static double orc_update_value(const orc_grid *g, const double *t, const double *r,
                               const double *c, int64_t idx)
{
    double a[3];
    orc_axis_minima(g, t, idx, a);
    return orc_dbar(a, g->D, r[idx], c[idx]);
}

/* Boundary nodes (sources): t := t0, duplicates keep the smallest t0. */
static void orc_init_field(const orc_grid *g, double *t, unsigned char *is_src,
                           const int64_t *src_idx, const double *src_t, int64_t nsrc)
{
    for (int64_t i = 0; i < g->N; ++i) { t[i] = ORC_INF; is_src[i] = 0; }
    for (int64_t s = 0; s < nsrc; ++s) {
        int64_t i = src_idx[s];
        double t0 = src_t ? src_t[s] : 0.0;
        if (!is_src[i] || t0 < t[i]) t[i] = t0;
        is_src[i] = 1;
    }
}

static void orc_constants(const orc_grid *g, const double *v, double h, double *r, double *c)
{
    for (int64_t i = 0; i < g->N; ++i) {
        r[i] = h / v[i];
        c[i] = r[i] * r[i];
    }
}

typedef struct {
    int64_t pops;          /* heap pops that were not stale */
    int64_t stale;         /* stale heap entries skipped */
    int64_t evals;         /* evaluations of the update operator */
    int64_t decreases;     /* evaluations that lowered a value */
    int64_t increases;     /* evaluations that would raise a value (must be 0) */
    int64_t order_breaks;  /* pops whose key is below the previous pop (must be 0) */
    int64_t sweeps;        /* sweeps of the topology-driven solvers */
} orc_stats;

/* ---------------------------------------------------------------------------
 * Fast marching method (Algorithm 2) with a binary heap.  Pop the smallest
 * entry, skip it if stale (its key is no longer the cell's value), update
 * every in-grid non-source neighbour and push it when its value decreased.
 * ------------------------------------------------------------------------- */

typedef struct { double key; int64_t idx; } orc_heap_item;
typedef struct { orc_heap_item *v; int64_t n, cap; } orc_heap;

static int heap_push(orc_heap *h, double key, int64_t idx)
{
    if (h->n == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        orc_heap_item *nv = (orc_heap_item *)realloc(h->v, (size_t)nc * sizeof(orc_heap_item));
        if (!nv) return -1;
        h->v = nv; h->cap = nc;
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->v[p].key <= key) break;
        h->v[i] = h->v[p];
        i = p;
    }
    h->v[i].key = key; h->v[i].idx = idx;
    return 0;
}

static orc_heap_item heap_pop(orc_heap *h)
{
    orc_heap_item top = h->v[0];
    orc_heap_item last = h->v[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        double mk = last.key;
        if (l < h->n && h->v[l].key < mk) { m = l; mk = h->v[l].key; }
        if (r < h->n && h->v[r].key < mk) { m = r; }
        if (m == i) break;
        h->v[i] = h->v[m];
        i = m;
    }
    if (h->n > 0) h->v[i] = last;
    return top;
}

/* Returns 0 on success, -1 on bad arguments or allocation failure. */
int orc_fmm(int ndim, const int64_t *dims, const double *v, double h,
            const int64_t *src_idx, const double *src_t, int64_t nsrc,
            double *t, orc_stats *st)
{
    orc_grid g;
    if (orc_grid_make(&g, ndim, dims)) return -1;
    orc_stats s = {0};
    double *r = (double *)malloc((size_t)g.N * sizeof(double));
    double *c = (double *)malloc((size_t)g.N * sizeof(double));
    unsigned char *is_src = (unsigned char *)malloc((size_t)g.N);
    orc_heap hp = {0};
    if (!r || !c || !is_src) { free(r); free(c); free(is_src); return -1; }
    orc_constants(&g, v, h, r, c);
    orc_init_field(&g, t, is_src, src_idx, src_t, nsrc);
    for (int64_t k = 0; k < nsrc; ++k) {
        int64_t i = src_idx[k];
        if (heap_push(&hp, t[i], i)) goto fail;
    }
    double last_key = -ORC_INF;
    while (hp.n > 0) {
        orc_heap_item it = heap_pop(&hp);
        if (it.key > t[it.idx]) { s.stale++; continue; }
        s.pops++;
        if (it.key < last_key) s.order_breaks++;
        last_key = it.key;
        int64_t rem = it.idx;
        for (int k = 0; k < g.D; ++k) {
            int64_t coord = rem % g.n[k];
            rem /= g.n[k];
            for (int side = 0; side < 2; ++side) {
                int64_t m;
                if (side == 0) { if (coord == 0) continue; m = it.idx - g.s[k]; }
                else { if (coord + 1 == g.n[k]) continue; m = it.idx + g.s[k]; }
                if (is_src[m]) continue;
                double tau = orc_update_value(&g, t, r, c, m);
                s.evals++;
                if (tau < t[m]) {
                    t[m] = tau;
                    s.decreases++;
                    if (heap_push(&hp, tau, m)) goto fail;
                } else if (tau > t[m]) {
                    s.increases++;
                }
            }
        }
    }
    free(hp.v); free(r); free(c); free(is_src);
    if (st) *st = s;
    return 0;
fail:
    free(hp.v); free(r); free(c); free(is_src);
    return -1;
}

/* ---------------------------------------------------------------------------
 * Topology-driven solvers: Algorithm 4 (every node, in index order, until a
 * sweep changes nothing) and Algorithm 5 (the fast sweeping method: the
 * 2^D alternating index orders, repeated until a full round changes nothing).
 * Brute force, for tiny grids.  mode 0 = Algorithm 4, mode 1 = Algorithm 5.
 * ------------------------------------------------------------------------- */

static int orc_sweep_once(const orc_grid *g, double *t, const double *r, const double *c,
                          const unsigned char *is_src, unsigned dirmask, orc_stats *s)
{
    int changed = 0;
    int64_t nz = g->D == 3 ? g->n[2] : 1;
    int64_t ny = g->D >= 2 ? g->n[1] : 1;
    int64_t nx = g->n[0];
    for (int64_t kz = 0; kz < nz; ++kz) {
        int64_t z = (dirmask & 4u) ? nz - 1 - kz : kz;
        for (int64_t ky = 0; ky < ny; ++ky) {
            int64_t y = (dirmask & 2u) ? ny - 1 - ky : ky;
            for (int64_t kx = 0; kx < nx; ++kx) {
                int64_t x = (dirmask & 1u) ? nx - 1 - kx : kx;
                int64_t idx = x + y * nx + z * nx * ny;
                if (is_src[idx]) continue;
                double tau = orc_update_value(g, t, r, c, idx);
                s->evals++;
                if (tau != t[idx]) {
                    if (tau > t[idx]) s->increases++;
                    t[idx] = tau;
                    s->decreases++;
                    changed = 1;
                }
            }
        }
    }
    return changed;
}

int orc_sweep(int ndim, const int64_t *dims, const double *v, double h,
              const int64_t *src_idx, const double *src_t, int64_t nsrc,
              int mode, double *t, orc_stats *st)
{
    orc_grid g;
    if (orc_grid_make(&g, ndim, dims)) return -1;
    orc_stats s = {0};
    double *r = (double *)malloc((size_t)g.N * sizeof(double));
    double *c = (double *)malloc((size_t)g.N * sizeof(double));
    unsigned char *is_src = (unsigned char *)malloc((size_t)g.N);
    if (!r || !c || !is_src) { free(r); free(c); free(is_src); return -1; }
    orc_constants(&g, v, h, r, c);
    orc_init_field(&g, t, is_src, src_idx, src_t, nsrc);
    unsigned ndirs = mode == 1 ? (1u << g.D) : 1u;
    for (;;) {
        int changed = 0;
        for (unsigned d = 0; d < ndirs; ++d) {
            changed |= orc_sweep_once(&g, t, r, c, is_src, mode == 1 ? d : 0u, &s);
            s.sweeps++;
        }
        if (!changed) break;
    }
    free(r); free(c); free(is_src);
    if (st) *st = s;
    return 0;
}

/* Relaxation in a caller-given cell order (Theorem 1: any order of
 * nontrivial updates ends at the same fixed point).  Passes over perm[]
 * repeat until one changes nothing.  The order is an input, drawn by the
 * caller. */
int orc_relax_order(int ndim, const int64_t *dims, const double *v, double h,
                    const int64_t *src_idx, const double *src_t, int64_t nsrc,
                    const int64_t *perm, int64_t nperm, double *t, orc_stats *st)
{
    orc_grid g;
    if (orc_grid_make(&g, ndim, dims)) return -1;
    orc_stats s = {0};
    double *r = (double *)malloc((size_t)g.N * sizeof(double));
    double *c = (double *)malloc((size_t)g.N * sizeof(double));
    unsigned char *is_src = (unsigned char *)malloc((size_t)g.N);
    if (!r || !c || !is_src) { free(r); free(c); free(is_src); return -1; }
    orc_constants(&g, v, h, r, c);
    orc_init_field(&g, t, is_src, src_idx, src_t, nsrc);
    for (;;) {
        int changed = 0;
        for (int64_t p = 0; p < nperm; ++p) {
            int64_t idx = perm[p];
            if (idx < 0 || idx >= g.N || is_src[idx]) continue;
            double tau = orc_update_value(&g, t, r, c, idx);
            s.evals++;
            if (tau != t[idx]) {
                if (tau > t[idx]) s.increases++;
                t[idx] = tau;
                s.decreases++;
                changed = 1;
            }
        }
        s.sweeps++;
        if (!changed) break;
    }
    free(r); free(c); free(is_src);
    if (st) *st = s;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Fixed-point residual (Table 3): re-apply the operator at every non-source
 * cell using the final values of its neighbours.  Writes the largest
 * relative difference |t - D(n,t)(n)| / t over finite cells to *max_rel and
 * returns the number of cells where the re-applied value differs from t at
 * all (0 for the exact fixed point), plus source cells whose value is not
 * their t0.  The operator is d-bar (form 0) or, in 2D, Algorithm 1 with the
 * explicit root d-tilde (form 1) or d-hat (form 2): the residual of a field
 * computed with that form, as Table 3 measures it.  Returns -1 on bad
 * arguments.
 * ------------------------------------------------------------------------- */
int64_t orc_residual_form(int form, int ndim, const int64_t *dims, const double *v, double h,
                          const int64_t *src_idx, const double *src_t, int64_t nsrc,
                          const double *t, double *max_rel)
{
    if (form != 0 && ndim != 2) return -1;
    orc_grid g;
    if (orc_grid_make(&g, ndim, dims)) return -1;
    unsigned char *is_src = (unsigned char *)calloc((size_t)g.N, 1);
    double *t0 = (double *)malloc((size_t)g.N * sizeof(double));
    if (!is_src || !t0) { free(is_src); free(t0); return -1; }
    for (int64_t s = 0; s < nsrc; ++s) {
        int64_t i = src_idx[s];
        double v0 = src_t ? src_t[s] : 0.0;
        if (!is_src[i] || v0 < t0[i]) t0[i] = v0;
        is_src[i] = 1;
    }
    int64_t bad = 0;
    double worst = 0.0;
    for (int64_t i = 0; i < g.N; ++i) {
        if (is_src[i]) {
            if (t[i] != t0[i]) bad++;
            continue;
        }
        double r = h / v[i];
        double c = r * r;
        double a[3];
        orc_axis_minima(&g, t, i, a);
        double tau = form == 0 ? orc_dbar(a, g.D, r, c) : orc_update_form(form, v[i], h, a[0], a[1]);
        if (tau != t[i]) {
            bad++;
            if (t[i] < ORC_INF && tau < ORC_INF && t[i] > 0.0) {
                double rel = fabs(t[i] - tau) / t[i];
                if (rel > worst) worst = rel;
            } else {
                worst = ORC_INF;
            }
        }
    }
    free(is_src); free(t0);
    if (max_rel) *max_rel = worst;
    return bad;
}

int64_t orc_residual(int ndim, const int64_t *dims, const double *v, double h,
                     const int64_t *src_idx, const double *src_t, int64_t nsrc,
                     const double *t, double *max_rel)
{
    return orc_residual_form(0, ndim, dims, v, h, src_idx, src_t, nsrc, t, max_rel);
}

/* ---------------------------------------------------------------------------
 * Adjoint of the fixed point (traveltime tomography).  Not in the paper: the
 * derivative of the real-arithmetic local equations at the computed field.
 * For a reached non-source cell n with axis minima a_k and the active axes
 * A(n) = {k : a_k < t_n} (both neighbours of an axis off-grid or at +inf: not
 * active), the local equation sum_{k in A} (t_n - a_k)^2 = h^2 s_n^2 with
 * slowness s = 1/v gives
 *   dt_n = [ sum_{k in A} (t_n - a_k) da_k + h^2 s_n ds_n ] / S_n,
 *   S_n  = sum_{k in A} (t_n - a_k)      (terms summed in axis order x, y, z),
 * and a_k is the neighbour holding the axis minimum (both neighbours, weight
 * 1/2 each, when they are equal).  For a loss L(t) with g = dL/dt:
 *   lambda_n = g_n + sum over downwind neighbours m of lambda_m * w(m, n),
 *   w(m, n)  = fl(fl(t_m - t_n) / S_m), halved when n shares the axis minimum
 *              of m with m's other neighbour on that axis,
 *   dL/ds_n  = lambda_n * fl(fl(fl(h*h) * s_n) / S_n),  s_n = fl(1/v_n),
 * with the downwind neighbours taken in the fixed order x-, x+, y-, y+, z-, z+
 * and every operation separately rounded.  Sources and unreached cells get
 * dL/ds = 0.  lambda is computed in decreasing t (every downwind neighbour has
 * a larger t).  Returns 0, or -1 on bad arguments / allocation failure.
 * ------------------------------------------------------------------------- */

typedef struct { double t; int64_t idx; } orc_tsort;

static int orc_tsort_desc(const void *pa, const void *pb)
{
    const orc_tsort *a = (const orc_tsort *)pa, *b = (const orc_tsort *)pb;
    if (a->t > b->t) return -1;
    if (a->t < b->t) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* S_n over the active axes of a reached non-source cell (0 if none). */
static double orc_upwind_sum(const orc_grid *g, const double *t, int64_t n)
{
    double a[3];
    orc_axis_minima(g, t, n, a);
    double S = 0.0;
    for (int k = 0; k < g->D; ++k)
        if (a[k] < t[n]) S = S + (t[n] - a[k]);
    return S;
}

/* Weight of neighbour u (at offset side along axis k of m) in dt_m, or 0. */
static double orc_weight(const orc_grid *g, const double *t, const unsigned char *is_src,
                         int64_t m, int k, int64_t u)
{
    if (is_src[m] || !(t[m] < ORC_INF)) return 0.0;
    double a[3];
    orc_axis_minima(g, t, m, a);
    if (!(a[k] < t[m]) || t[u] != a[k]) return 0.0;
    double S = orc_upwind_sum(g, t, m);
    double w = (t[m] - t[u]) / S;
    /* the other neighbour of m on axis k, if in-grid, equal to the minimum */
    int64_t rem = m, coord = 0;
    for (int j = 0; j <= k; ++j) { coord = rem % g->n[j]; rem /= g->n[j]; }
    int64_t other = (u < m) ? m + g->s[k] : m - g->s[k];
    int in = (u < m) ? (coord + 1 < g->n[k]) : (coord > 0);
    if (in && t[other] == t[u]) w = w * 0.5;
    return w;
}

int orc_adjoint(int ndim, const int64_t *dims, const double *v, double h,
                const int64_t *src_idx, int64_t nsrc, const double *t, const double *dL_dt,
                double *lambda, double *dL_ds)
{
    orc_grid g;
    if (orc_grid_make(&g, ndim, dims)) return -1;
    unsigned char *is_src = (unsigned char *)calloc((size_t)g.N, 1);
    orc_tsort *order = (orc_tsort *)malloc((size_t)g.N * sizeof(orc_tsort));
    if (!is_src || !order) { free(is_src); free(order); return -1; }
    for (int64_t s = 0; s < nsrc; ++s) is_src[src_idx[s]] = 1;
    int64_t nr = 0;
    for (int64_t i = 0; i < g.N; ++i) {
        lambda[i] = 0.0;
        dL_ds[i] = 0.0;
        if (t[i] < ORC_INF) { order[nr].t = t[i]; order[nr].idx = i; ++nr; }
    }
    qsort(order, (size_t)nr, sizeof(orc_tsort), orc_tsort_desc);
    double hh = h * h;
    for (int64_t q = 0; q < nr; ++q) {
        int64_t n = order[q].idx;
        double lam = dL_dt[n];
        int64_t rem = n;
        for (int k = 0; k < g.D; ++k) {
            int64_t coord = rem % g.n[k];
            rem /= g.n[k];
            for (int side = 0; side < 2; ++side) {
                int64_t m;
                if (side == 0) { if (coord == 0) continue; m = n - g.s[k]; }
                else { if (coord + 1 == g.n[k]) continue; m = n + g.s[k]; }
                if (!(t[m] > t[n])) continue;              /* downwind only */
                double w = orc_weight(&g, t, is_src, m, k, n);
                if (w != 0.0) lam = lam + lambda[m] * w;
            }
        }
        lambda[n] = lam;
        if (!is_src[n]) {
            double S = orc_upwind_sum(&g, t, n);
            if (S > 0.0) {
                double s = 1.0 / v[n];
                dL_ds[n] = lam * ((hh * s) / S);
            }
        }
    }
    free(is_src); free(order);
    return 0;
}
