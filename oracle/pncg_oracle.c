/*
 * FP64 CPU oracle for the Jacobi-preconditioned nonlinear conjugate gradient (PNCG) solver of
 * Shen, Cai, Bi, Lv, "Preconditioned Nonlinear Conjugate Gradient Method for Real-time Interior-point
 * Hyperelasticity", SIGGRAPH 2024 (arXiv 2405.08001).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference the CUDA library is checked against.  Only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark load it; the library never does,
 * and the two share no code.  Everything is double precision, serial, and summed in index order.
 *
 * What it computes, by paper section:
 *   - incremental potential E(x) = 1/2 (x - xt)^T M (x - xt) + h^2 Psi(x) + kappa sum_C b(d_k)   (Sec. 3, Eq. E)
 *   - Neo-Hookean Psi = mu/2 (I2 - 3) - mu log I3 + lambda/2 (log I3)^2                        (Sec. 3.1)
 *     and the other densities of the invariants I1 = tr(S), I2, I3: stable Neo-Hookean, fixed corotated,
 *     as-rigid-as-possible (the materials of Table 1), I1 through the polar decomposition F = R S   (Sec. 3.1)
 *     with its gradient, its Hessian diagonal and p^T H p through the six-term split
 *     sum_i (Psi_ii h_i + Psi_i h_{i+3}) using vec(dF/dx) as an explicit 9x12 matrix            (Sec. 3.1)
 *   - the log barrier b(d) and its gradient / diagonal / p^T H p through t and c_0..c_3          (Sec. 3.2, Eqs. 8-13)
 *   - the point-triangle and edge-edge distances as minimisations over the coefficient sets      (Sec. 3.2, Eqs. PT, EE)
 *   - one PNCG iteration and a whole time step                                                    (Sec. 4, Algorithm 1)
 *   - preconditioned Polak-Ribiere+ (default) or Dai-Kou beta                                    (Sec. 4.1-4.2)
 *   - the single-pass step alpha = min(dhat / (2 ||p||_inf), -g^T p / p^T H p)                   (Sec. 4.3, Eqs. upper, alpha)
 *   - the rest-pose exclusion of self-collision pairs closer than 1.5 dhat                        (Sec. 5.1)
 *   - per-object splitting: each object its own beta, direction and step                         (Sec. 5.2)
 *   - differentiation, which the paper does not have: H v as the vector form of p^T H p, and the reverse of one
 *     time step read as the exact minimiser of its potential (implicit function theorem; linear CG on H v)
 *
 * Readings where the paper is silent (each one is also taken by the CUDA library):
 *   - Psi(x) = sum_e V_e Psi_NH(F_e), F = Ds Dm^-1 with D = [x1-x0, x2-x0, x3-x0]; mu = E/(2(1+nu)),
 *     lambda = E nu / ((1+nu)(1-2nu)); lumped mass m_v = sum_e rho V_e / 4.
 *   - the barrier Hessian freezes the closest-point coefficients c (Sec. 3.2 states d2t/dx2 = 0).
 *   - closest points: PT interior projection (2x2 normal equations), else the three clamped point-edge cases;
 *     EE interior solution (2x2), else the four clamped point-edge cases; ties keep the first case in that order.
 *   - preconditioner P_ii = 1 / diag_ii, the Jacobi preconditioner of Sec. 4.2, wherever diag_ii > 1e-3 m_v; the
 *     inertia diagonal alone, P_ii = 1 / m_v, where diag_ii <= 1e-3 m_v.  The barrier term (b'/d) c_i^2 of Eq. 9-10
 *     is negative (b' < 0 inside dhat), so on contact vertices diag(H) can reach zero or fall below it, where
 *     diag(H)^-1 is unbounded or negative (not a preconditioner); kinematic vertices get P = 0, g = 0.
 *   - PR+ beta = max(0, g1^T P1 (g1 - g0) / (g0^T P0 g0)); restart (beta = 0) when g^T p >= 0 after forming p.
 *   - ||p||_inf in the step cap is the largest per-vertex Euclidean length (the cap bounds vertex displacement
 *     by dhat/2, Sec. 4.3); the largest absolute component is an option.
 *   - if p^T H p <= 0 or the Newton step is not finite, alpha = alpha_upper.
 *   - a vertex-half-space barrier d = n.x - o with the same b, kappa and dhat stands in for a ground plane.
 *   - contacts are only between surface primitives (faces used by exactly one tet, their edges and vertices).
 *   - "self-collision" in the rest-pose exclusion means both primitives lie in one object, an object being a
 *     connected component of the tet mesh; pairs between different objects are never excluded.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_INVERTED 2
#define OR_ERR_PENETRATION 3
#define OR_ERR_NONFINITE 4
#define OR_ERR_OOM 5

#define OR_PT 0
#define OR_EE 1

static char g_err[256] = "";
static void set_err(const char *m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char *or_last_error(void) { return g_err; }

typedef struct {
    int32_t nv, nt;
    const double *rest_x;          /* [nv*3] */
    const int32_t *tets;           /* [nt*4] */
    const double *youngs_per_tet;  /* [nt] or NULL */
    double youngs, poisson, density;
    double h, dhat, kappa;
    double gravity[3];
    int32_t has_plane;
    double plane_n[3];
    double plane_o;
    const uint8_t *fixed;          /* [nv] or NULL */
    int32_t beta_rule;             /* 0 = PR+, 1 = DK */
    int32_t pnorm;                 /* 0 = max vertex 2-norm, 1 = max abs component */
    double excl_factor;            /* rest-pose exclusion radius in units of dhat (Sec. 5.1 uses 1.5) */
    int32_t model;                 /* energy density: OR_NH, OR_SNH, OR_FCR, OR_ARAP (Sec. 3.1, Table 1) */
} or_params;

/* energy densities in the invariants I1 = tr(S) (F = R S), I2 = tr(F^T F), I3 = det F of Sec. 3.1:
 *   NH   mu/2 (I2 - 3) - mu log I3 + lambda/2 (log I3)^2        (the paper's Neo-Hookean)
 *   SNH  mu/2 (I2 - 3) - mu (I3 - 1) + lambda/2 (I3 - 1)^2       (stable Neo-Hookean)
 *   FCR  mu (I2 - 2 I1 + 3) + lambda/2 (I3 - 1)^2               (fixed corotated: mu |F - R|^2 + ...)
 *   ARAP mu (I2 - 2 I1 + 3)                                      (as-rigid-as-possible: mu |F - R|^2) */
#define OR_NH 0
#define OR_SNH 1
#define OR_FCR 2
#define OR_ARAP 3

typedef struct {
    int32_t type;       /* OR_PT: v[0] point, v[1..3] triangle; OR_EE: v[0]-v[1] and v[2]-v[3] */
    int32_t v[4];
    int32_t a, b;       /* primitive ids: (vertex, triangle) or (edge, edge) with a < b */
    double d, c[4], t[3];
} or_pair;

typedef struct {
    or_params p;
    double *X;          /* rest positions */
    int32_t *tet;
    double *Dminv;      /* [nt][3][3] row-major */
    double *vol, *mu, *lam;
    double *mass;
    uint8_t *fixed;
    int32_t nf, ne, ns;
    int32_t *tri, *edge, *svert;
    double cell;        /* grid cell size for the contact search */
    int32_t *obj;       /* connected component (object) of each vertex */
    int32_t nexcl;
    uint64_t *excl;     /* sorted keys of excluded pairs */
    double plane_n[3];
} or_model;

typedef struct {
    int32_t k;
    double dE0;
    double beta, gp, pHp, pmax, alpha_bar, alpha_up, alpha, dE;
    int32_t restarted, capped, n_active, n_plane;
} or_ncg_scalars;

/* ------------------------------------------------------------------------------------------------ small linear algebra */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double det3(const double M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}
static int inv3(const double M[3][3], double I[3][3])
{
    double d = det3(M);
    if (!(fabs(d) > 0.0)) return 0;
    I[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / d;
    I[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / d;
    I[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / d;
    I[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / d;
    I[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / d;
    I[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / d;
    I[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / d;
    I[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / d;
    I[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / d;
    return 1;
}

/* ------------------------------------------------------------------------------------------------ barrier (Eq. barrier) */

/* b(d) = -(d - dhat)^2 log(d / dhat) on 0 < d < dhat, 0 for d >= dhat, with its first two derivatives in d. */
void or_barrier_fn(double d, double dhat, double *out3)
{
    if (d >= dhat) { out3[0] = out3[1] = out3[2] = 0.0; return; }
    double r = d - dhat, L = log(d / dhat);
    out3[0] = -r * r * L;
    out3[1] = -2.0 * r * L - r * r / d;
    out3[2] = -2.0 * L - 4.0 * r / d + r * r / (d * d);
}

/* ------------------------------------------------------------------------------------------------ distances (Sec. 3.2) */

/* closest point of segment a-b to q: parameter u in [0,1] of a + u (b - a); returns the squared distance */
static double point_segment(const double *q, const double *a, const double *b, double *u)
{
    double ab[3], aq[3];
    sub3(b, a, ab);
    sub3(q, a, aq);
    double L2 = dot3(ab, ab);
    double s = L2 > 0.0 ? dot3(aq, ab) / L2 : 0.0;
    if (s < 0.0) s = 0.0;
    if (s > 1.0) s = 1.0;
    double r[3] = {aq[0] - s * ab[0], aq[1] - s * ab[1], aq[2] - s * ab[2]};
    *u = s;
    return dot3(r, r);
}

/*
 * Distance between primitives as the norm of t = sum c_i x_i, minimised over the paper's coefficient sets:
 *   PT: c0 = 1, c1..c3 <= 0, c1 + c2 + c3 = -1   (x0 the point, x1 x2 x3 the triangle)
 *   EE: c0, c1 >= 0, c0 + c1 = 1, c2, c3 <= 0, c2 + c3 = -1   (edges x0-x1 and x2-x3)
 * x is [4][3].  Writes c[4] and t[3]; returns d.
 */
double or_pair_geometry(int32_t type, const double *x, double *c, double *t)
{
    const double *x0 = x, *x1 = x + 3, *x2 = x + 6, *x3 = x + 9;
    double best = INFINITY;
    double cc[4];
    if (type == OR_PT) {
        double e1[3], e2[3], r[3];
        sub3(x2, x1, e1);
        sub3(x3, x1, e2);
        sub3(x0, x1, r);
        double a = dot3(e1, e1), b = dot3(e1, e2), cq = dot3(e2, e2);
        double det = a * cq - b * b;
        if (det > 1e-12 * a * cq) {
            double p = dot3(r, e1), q = dot3(r, e2);
            double be = (cq * p - b * q) / det, ga = (a * q - b * p) / det;
            if (be >= 0.0 && ga >= 0.0 && be + ga <= 1.0) {
                cc[0] = 1.0; cc[1] = -(1.0 - be - ga); cc[2] = -be; cc[3] = -ga;
                memcpy(c, cc, sizeof cc);
                best = -1.0;
            }
        }
        if (best != -1.0) {
            const double *tri[3] = {x1, x2, x3};
            for (int k = 0; k < 3; ++k) {
                int i = k, j = (k + 1) % 3;
                double u;
                double d2 = point_segment(x0, tri[i], tri[j], &u);
                if (d2 < best) {
                    best = d2;
                    cc[0] = 1.0; cc[1] = cc[2] = cc[3] = 0.0;
                    cc[1 + i] = -(1.0 - u);
                    cc[1 + j] = -u;
                    memcpy(c, cc, sizeof cc);
                }
            }
        }
    } else {
        double e0[3], e1[3], r[3];
        sub3(x1, x0, e0);
        sub3(x3, x2, e1);
        sub3(x0, x2, r);
        double a = dot3(e0, e0), b = dot3(e0, e1), cq = dot3(e1, e1), dd = dot3(e0, r), ee = dot3(e1, r);
        double det = a * cq - b * b;
        if (det > 1e-12 * a * cq) {
            double s = (b * ee - cq * dd) / det, u = (a * ee - b * dd) / det;
            if (s >= 0.0 && s <= 1.0 && u >= 0.0 && u <= 1.0) {
                c[0] = 1.0 - s; c[1] = s; c[2] = -(1.0 - u); c[3] = -u;
                best = -1.0;
            }
        }
        if (best != -1.0) {
            double u, d2;
            /* s = 0: x0 against edge x2-x3 */
            d2 = point_segment(x0, x2, x3, &u);
            if (d2 < best) { best = d2; c[0] = 1.0; c[1] = 0.0; c[2] = -(1.0 - u); c[3] = -u; }
            /* s = 1: x1 against edge x2-x3 */
            d2 = point_segment(x1, x2, x3, &u);
            if (d2 < best) { best = d2; c[0] = 0.0; c[1] = 1.0; c[2] = -(1.0 - u); c[3] = -u; }
            /* u = 0: x2 against edge x0-x1 */
            d2 = point_segment(x2, x0, x1, &u);
            if (d2 < best) { best = d2; c[0] = 1.0 - u; c[1] = u; c[2] = -1.0; c[3] = 0.0; }
            /* u = 1: x3 against edge x0-x1 */
            d2 = point_segment(x3, x0, x1, &u);
            if (d2 < best) { best = d2; c[0] = 1.0 - u; c[1] = u; c[2] = 0.0; c[3] = -1.0; }
        }
    }
    for (int a = 0; a < 3; ++a) t[a] = c[0] * x0[a] + c[1] * x1[a] + c[2] * x2[a] + c[3] * x3[a];
    return sqrt(dot3(t, t));
}

/* ------------------------------------------------------------------------------------------------ sorting helpers */

static int cmp_i3(const void *pa, const void *pb)
{
    const int32_t *a = pa, *b = pb;
    for (int k = 0; k < 3; ++k) if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
    return 0;
}
static int cmp_i2(const void *pa, const void *pb)
{
    const int32_t *a = pa, *b = pb;
    for (int k = 0; k < 2; ++k) if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
    return 0;
}
static int cmp_u64(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}
static void sort3(int32_t *v)
{
    int32_t t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

static uint64_t pair_key(int32_t type, int32_t a, int32_t b)
{
    return ((uint64_t)type << 62) | ((uint64_t)(uint32_t)a << 31) | (uint64_t)(uint32_t)b;
}

/* ------------------------------------------------------------------------------------------------ contact search */

typedef struct { uint64_t key; int32_t prim; } cell_entry;

static int cmp_cell(const void *pa, const void *pb)
{
    const cell_entry *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->prim < b->prim ? -1 : (a->prim > b->prim ? 1 : 0);
}

#define CELL_OFF (1 << 20)
static uint64_t cell_key3(int64_t i, int64_t j, int64_t k)
{
    return ((uint64_t)(i + CELL_OFF) << 42) | ((uint64_t)(j + CELL_OFF) << 21) | (uint64_t)(k + CELL_OFF);
}

typedef struct { or_pair *v; int32_t n, cap; } pair_list;

static int push_pair(pair_list *L, const or_pair *p)
{
    if (L->n == L->cap) {
        int32_t nc = L->cap ? 2 * L->cap : 256;
        or_pair *nv = realloc(L->v, (size_t)nc * sizeof(or_pair));
        if (!nv) return 0;
        L->v = nv;
        L->cap = nc;
    }
    L->v[L->n++] = *p;
    return 1;
}

static int cmp_pair(const void *pa, const void *pb)
{
    const or_pair *a = pa, *b = pb;
    if (a->type != b->type) return a->type < b->type ? -1 : 1;
    if (a->a != b->a) return a->a < b->a ? -1 : 1;
    return a->b < b->b ? -1 : (a->b > b->b ? 1 : 0);
}

static int excluded(const or_model *m, int32_t type, int32_t a, int32_t b)
{
    if (m->nexcl == 0) return 0;
    uint64_t k = pair_key(type, a, b);
    return bsearch(&k, m->excl, (size_t)m->nexcl, sizeof(uint64_t), cmp_u64) != NULL;
}

static void gather4(const double *x, const int32_t *v, double *out)
{
    for (int i = 0; i < 4; ++i) memcpy(out + 3 * i, x + 3 * (size_t)v[i], 3 * sizeof(double));
}

/* test one candidate; append it when d < thr (and not excluded when use_excl) */
static int try_pair(const or_model *m, const double *x, int32_t type, int32_t a, int32_t b, double thr,
                    int use_excl, pair_list *L)
{
    or_pair P;
    P.type = type;
    P.a = a;
    P.b = b;
    if (type == OR_PT) {
        P.v[0] = m->svert[a];
        P.v[1] = m->tri[3 * b]; P.v[2] = m->tri[3 * b + 1]; P.v[3] = m->tri[3 * b + 2];
        if (P.v[0] == P.v[1] || P.v[0] == P.v[2] || P.v[0] == P.v[3]) return 1;
    } else {
        P.v[0] = m->edge[2 * a]; P.v[1] = m->edge[2 * a + 1];
        P.v[2] = m->edge[2 * b]; P.v[3] = m->edge[2 * b + 1];
        if (P.v[0] == P.v[2] || P.v[0] == P.v[3] || P.v[1] == P.v[2] || P.v[1] == P.v[3]) return 1;
    }
    double xs[12];
    gather4(x, P.v, xs);
    P.d = or_pair_geometry(type, xs, P.c, P.t);
    if (!(P.d < thr)) return 1;
    if (use_excl && m->obj[P.v[0]] == m->obj[P.v[2]] && excluded(m, type, a, b)) return 1;
    return push_pair(L, &P);
}

static void prim_box(const double *x, const int32_t *v, int nvert, double lo[3], double hi[3])
{
    for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int i = 0; i < nvert; ++i)
        for (int a = 0; a < 3; ++a) {
            double c = x[3 * (size_t)v[i] + a];
            if (c < lo[a]) lo[a] = c;
            if (c > hi[a]) hi[a] = c;
        }
}

/*
 * All surface pairs with d < thr: PT (vertex not in the triangle) and EE (edges sharing no vertex), sorted by
 * (type, a, b).  brute = 1 tests every pair; otherwise a uniform grid (sorted cell lists) culls the candidates.
 */
static int find_pairs(const or_model *m, const double *x, double thr, int use_excl, int brute, pair_list *L)
{
    L->n = 0;
    double s = m->cell;
    if (!brute) {
        for (int32_t i = 0; i < m->p.nv; ++i)
            for (int a = 0; a < 3; ++a) {
                double q = x[3 * (size_t)i + a] / s;
                if (!(fabs(q) < (double)(CELL_OFF - 4))) brute = 1;
            }
    }
    if (brute) {
        for (int32_t a = 0; a < m->ns; ++a)
            for (int32_t b = 0; b < m->nf; ++b)
                if (!try_pair(m, x, OR_PT, a, b, thr, use_excl, L)) return OR_ERR_OOM;
        for (int32_t a = 0; a < m->ne; ++a)
            for (int32_t b = a + 1; b < m->ne; ++b)
                if (!try_pair(m, x, OR_EE, a, b, thr, use_excl, L)) return OR_ERR_OOM;
        qsort(L->v, (size_t)L->n, sizeof(or_pair), cmp_pair);
        return OR_OK;
    }
    /* grid over triangles (boxes inflated by thr); each surface vertex looks up its own cell */
    for (int pass = 0; pass < 2; ++pass) {
        int32_t nprim = pass == 0 ? m->nf : m->ne;
        int nvp = pass == 0 ? 3 : 2;
        const int32_t *pv = pass == 0 ? m->tri : m->edge;
        size_t cap = 1024, n = 0;
        cell_entry *E = malloc(cap * sizeof(cell_entry));
        if (!E) return OR_ERR_OOM;
        for (int32_t f = 0; f < nprim; ++f) {
            double lo[3], hi[3];
            prim_box(x, pv + (size_t)nvp * f, nvp, lo, hi);
            int64_t l[3], h[3];
            for (int a = 0; a < 3; ++a) { l[a] = (int64_t)floor((lo[a] - thr) / s); h[a] = (int64_t)floor((hi[a] + thr) / s); }
            for (int64_t i = l[0]; i <= h[0]; ++i)
                for (int64_t j = l[1]; j <= h[1]; ++j)
                    for (int64_t k = l[2]; k <= h[2]; ++k) {
                        if (n == cap) {
                            cap *= 2;
                            cell_entry *nE = realloc(E, cap * sizeof(cell_entry));
                            if (!nE) { free(E); return OR_ERR_OOM; }
                            E = nE;
                        }
                        E[n].key = cell_key3(i, j, k);
                        E[n].prim = f;
                        ++n;
                    }
        }
        qsort(E, n, sizeof(cell_entry), cmp_cell);
        if (pass == 0) {
            for (int32_t a = 0; a < m->ns; ++a) {
                const double *q = x + 3 * (size_t)m->svert[a];
                uint64_t key = cell_key3((int64_t)floor(q[0] / s), (int64_t)floor(q[1] / s), (int64_t)floor(q[2] / s));
                size_t lo = 0, hi = n;
                while (lo < hi) { size_t mid = (lo + hi) / 2; if (E[mid].key < key) lo = mid + 1; else hi = mid; }
                for (size_t e = lo; e < n && E[e].key == key; ++e)
                    if (!try_pair(m, x, OR_PT, a, E[e].prim, thr, use_excl, L)) { free(E); return OR_ERR_OOM; }
            }
        } else {
            int32_t *mark = malloc((size_t)(m->ne > 0 ? m->ne : 1) * sizeof(int32_t));
            if (!mark) { free(E); return OR_ERR_OOM; }
            for (int32_t e = 0; e < m->ne; ++e) mark[e] = -1;
            for (int32_t a = 0; a < m->ne; ++a) {
                double lo[3], hi[3];
                prim_box(x, m->edge + 2 * (size_t)a, 2, lo, hi);
                int64_t l[3], h[3];
                for (int c = 0; c < 3; ++c) { l[c] = (int64_t)floor(lo[c] / s); h[c] = (int64_t)floor(hi[c] / s); }
                for (int64_t i = l[0]; i <= h[0]; ++i)
                    for (int64_t j = l[1]; j <= h[1]; ++j)
                        for (int64_t k = l[2]; k <= h[2]; ++k) {
                            uint64_t key = cell_key3(i, j, k);
                            size_t lo2 = 0, hi2 = n;
                            while (lo2 < hi2) { size_t mid = (lo2 + hi2) / 2; if (E[mid].key < key) lo2 = mid + 1; else hi2 = mid; }
                            for (size_t e = lo2; e < n && E[e].key == key; ++e) {
                                int32_t b = E[e].prim;
                                if (b <= a || mark[b] == a) continue;
                                mark[b] = a;
                                if (!try_pair(m, x, OR_EE, a, b, thr, use_excl, L)) { free(mark); free(E); return OR_ERR_OOM; }
                            }
                        }
            }
            free(mark);
        }
        free(E);
    }
    qsort(L->v, (size_t)L->n, sizeof(or_pair), cmp_pair);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------------ model set-up */

void or_model_free(or_model *m)
{
    if (!m) return;
    free(m->X); free(m->tet); free(m->Dminv); free(m->vol); free(m->mu); free(m->lam); free(m->mass);
    free(m->fixed); free(m->tri); free(m->edge); free(m->svert); free(m->excl); free(m->obj);
    free(m);
}

or_model *or_model_new(const or_params *p)
{
    if (!p || p->nv <= 0 || p->nt <= 0 || !p->rest_x || !p->tets || !(p->h > 0) || !(p->dhat > 0) || p->kappa < 0 ||
        p->model < OR_NH || p->model > OR_ARAP) {
        set_err("invalid parameters");
        return NULL;
    }
    or_model *m = calloc(1, sizeof(or_model));
    if (!m) { set_err("out of memory"); return NULL; }
    m->p = *p;
    m->p.rest_x = NULL; m->p.tets = NULL; m->p.youngs_per_tet = NULL; m->p.fixed = NULL;
    int32_t nv = p->nv, nt = p->nt;
    m->X = malloc(sizeof(double) * 3 * (size_t)nv);
    m->tet = malloc(sizeof(int32_t) * 4 * (size_t)nt);
    m->Dminv = malloc(sizeof(double) * 9 * (size_t)nt);
    m->vol = malloc(sizeof(double) * (size_t)nt);
    m->mu = malloc(sizeof(double) * (size_t)nt);
    m->lam = malloc(sizeof(double) * (size_t)nt);
    m->mass = calloc((size_t)nv, sizeof(double));
    m->fixed = calloc((size_t)nv, 1);
    if (!m->X || !m->tet || !m->Dminv || !m->vol || !m->mu || !m->lam || !m->mass || !m->fixed) {
        set_err("out of memory"); or_model_free(m); return NULL;
    }
    memcpy(m->X, p->rest_x, sizeof(double) * 3 * (size_t)nv);
    memcpy(m->tet, p->tets, sizeof(int32_t) * 4 * (size_t)nt);
    if (p->fixed) memcpy(m->fixed, p->fixed, (size_t)nv);
    if (p->has_plane) {
        double L = sqrt(dot3(p->plane_n, p->plane_n));
        if (!(L > 0)) { set_err("zero plane normal"); or_model_free(m); return NULL; }
        for (int a = 0; a < 3; ++a) m->plane_n[a] = p->plane_n[a] / L;
    }
    for (int32_t e = 0; e < nt; ++e) {
        const int32_t *v = m->tet + 4 * (size_t)e;
        for (int i = 0; i < 4; ++i)
            if (v[i] < 0 || v[i] >= nv) { set_err("tet index out of range"); or_model_free(m); return NULL; }
        double Dm[3][3], Di[3][3];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) Dm[a][c] = m->X[3 * (size_t)v[c + 1] + a] - m->X[3 * (size_t)v[0] + a];
        double vol = det3(Dm) / 6.0;
        if (!(vol > 0.0) || !inv3(Dm, Di)) { set_err("tet with non-positive rest volume"); or_model_free(m); return NULL; }
        memcpy(m->Dminv + 9 * (size_t)e, Di, sizeof Di);
        m->vol[e] = vol;
        double E = p->youngs_per_tet ? p->youngs_per_tet[e] : p->youngs, nu = p->poisson;
        m->mu[e] = E / (2.0 * (1.0 + nu));
        m->lam[e] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        for (int i = 0; i < 4; ++i) m->mass[v[i]] += p->density * vol / 4.0;
    }
    /* surface: faces used by exactly one tet, their unique edges and their vertices */
    int32_t *F = malloc(sizeof(int32_t) * 12 * (size_t)nt);
    if (!F) { set_err("out of memory"); or_model_free(m); return NULL; }
    static const int fv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    for (int32_t e = 0; e < nt; ++e)
        for (int f = 0; f < 4; ++f) {
            int32_t *o = F + 3 * (4 * (size_t)e + f);
            for (int k = 0; k < 3; ++k) o[k] = m->tet[4 * (size_t)e + fv[f][k]];
            sort3(o);
        }
    qsort(F, 4 * (size_t)nt, 3 * sizeof(int32_t), cmp_i3);
    m->tri = malloc(sizeof(int32_t) * 12 * (size_t)nt);
    int32_t nf = 0;
    for (size_t i = 0; i < 4 * (size_t)nt;) {
        size_t j = i + 1;
        while (j < 4 * (size_t)nt && cmp_i3(F + 3 * i, F + 3 * j) == 0) ++j;
        if (j - i == 1) { memcpy(m->tri + 3 * (size_t)nf, F + 3 * i, 3 * sizeof(int32_t)); ++nf; }
        i = j;
    }
    free(F);
    m->nf = nf;
    int32_t *Ed = malloc(sizeof(int32_t) * 6 * (size_t)(nf > 0 ? nf : 1));
    for (int32_t f = 0; f < nf; ++f) {
        const int32_t *t = m->tri + 3 * (size_t)f;
        int32_t pr[3][2] = {{t[0], t[1]}, {t[1], t[2]}, {t[0], t[2]}};
        for (int k = 0; k < 3; ++k) { Ed[6 * (size_t)f + 2 * k] = pr[k][0]; Ed[6 * (size_t)f + 2 * k + 1] = pr[k][1]; }
    }
    qsort(Ed, 3 * (size_t)nf, 2 * sizeof(int32_t), cmp_i2);
    m->edge = malloc(sizeof(int32_t) * 6 * (size_t)(nf > 0 ? nf : 1));
    int32_t ne = 0;
    for (size_t i = 0; i < 3 * (size_t)nf; ++i)
        if (i == 0 || cmp_i2(Ed + 2 * i, Ed + 2 * (i - 1)) != 0) { memcpy(m->edge + 2 * (size_t)ne, Ed + 2 * i, 2 * sizeof(int32_t)); ++ne; }
    free(Ed);
    m->ne = ne;
    uint8_t *on = calloc((size_t)nv, 1);
    for (int32_t f = 0; f < nf; ++f) for (int k = 0; k < 3; ++k) on[m->tri[3 * (size_t)f + k]] = 1;
    m->svert = malloc(sizeof(int32_t) * (size_t)nv);
    int32_t ns = 0;
    for (int32_t i = 0; i < nv; ++i) if (on[i]) m->svert[ns++] = i;
    free(on);
    m->ns = ns;
    /* grid cell: mean rest surface edge length, at least dhat */
    double Lsum = 0.0;
    for (int32_t e = 0; e < ne; ++e) {
        double d[3];
        sub3(m->X + 3 * (size_t)m->edge[2 * e + 1], m->X + 3 * (size_t)m->edge[2 * e], d);
        Lsum += sqrt(dot3(d, d));
    }
    m->cell = ne > 0 ? Lsum / ne : 1.0;
    if (m->cell < p->dhat) m->cell = p->dhat;
    /* objects: connected components of the tet mesh (union-find over tet vertices) */
    m->obj = malloc(sizeof(int32_t) * (size_t)nv);
    if (!m->obj) { set_err("out of memory"); or_model_free(m); return NULL; }
    for (int32_t i = 0; i < nv; ++i) m->obj[i] = i;
    for (int32_t e = 0; e < nt; ++e)
        for (int k = 1; k < 4; ++k) {
            int32_t a = m->tet[4 * (size_t)e], b = m->tet[4 * (size_t)e + k];
            while (m->obj[a] != a) a = m->obj[a];
            while (m->obj[b] != b) b = m->obj[b];
            if (a != b) { if (a < b) m->obj[b] = a; else m->obj[a] = b; }
        }
    for (int32_t i = 0; i < nv; ++i) { int32_t r = i; while (m->obj[r] != r) r = m->obj[r]; m->obj[i] = r; }
    /* rest-pose exclusion (Sec. 5.1): self-collision pairs (both primitives in one object) closer than
       excl_factor * dhat at rest are never active */
    m->nexcl = 0;
    m->excl = NULL;
    if (p->excl_factor > 0) {
        pair_list L = {0};
        int st = find_pairs(m, m->X, p->excl_factor * p->dhat, 0, 0, &L);
        if (st != OR_OK) { free(L.v); set_err("out of memory"); or_model_free(m); return NULL; }
        m->excl = malloc(sizeof(uint64_t) * (size_t)(L.n > 0 ? L.n : 1));
        int32_t ne_ = 0;
        for (int32_t i = 0; i < L.n; ++i)
            if (m->obj[L.v[i].v[0]] == m->obj[L.v[i].v[2]]) m->excl[ne_++] = pair_key(L.v[i].type, L.v[i].a, L.v[i].b);
        m->nexcl = ne_;
        qsort(m->excl, (size_t)m->nexcl, sizeof(uint64_t), cmp_u64);
        free(L.v);
    }
    return m;
}

void or_model_sizes(const or_model *m, int32_t *out)
{
    out[0] = m->p.nv; out[1] = m->p.nt; out[2] = m->nf; out[3] = m->ne; out[4] = m->ns; out[5] = m->nexcl;
}

void or_model_arrays(const or_model *m, double *mass, double *vol, double *Dminv)
{
    if (mass) memcpy(mass, m->mass, sizeof(double) * (size_t)m->p.nv);
    if (vol) memcpy(vol, m->vol, sizeof(double) * (size_t)m->p.nt);
    if (Dminv) memcpy(Dminv, m->Dminv, sizeof(double) * 9 * (size_t)m->p.nt);
}

void or_surface(const or_model *m, int32_t *tri, int32_t *edge, int32_t *svert)
{
    if (tri) memcpy(tri, m->tri, sizeof(int32_t) * 3 * (size_t)m->nf);
    if (edge) memcpy(edge, m->edge, sizeof(int32_t) * 2 * (size_t)m->ne);
    if (svert) memcpy(svert, m->svert, sizeof(int32_t) * (size_t)m->ns);
}

/* ------------------------------------------------------------------------------------------------ Neo-Hookean (Sec. 3.1) */

/*
 * Per-tet quantities in the paper's notation.  J = vec(dF/dx) is 9x12 with vec() the column-wise flattening:
 * row 3b+a (entry F_ab), column 3i+a' (vertex i, component a'):  J = delta_{a a'} w_i[b], where
 * w_0 = -(sum of the rows of Dm^-1) and w_i = row i-1 of Dm^-1.
 */
typedef struct {
    double F[3][3];
    double J[9][12];
    double I1, I2, I3, logI3;
    double g1[9], g2[9], g3[9];   /* gradients of I1, I2 and I3 with respect to vec(F) */
    double H1[9][9];              /* Hessian of I1 (FCR, ARAP only; zero otherwise) */
    double H3[9][9];              /* Hessian of I3; H2 = 2 I */
    double Psi1, Psi2, Psi3, Psi11, Psi22, Psi33;
    double scale;                 /* h^2 V_e */
} tet_terms;

/*
 * Eigen-decomposition of a symmetric 3x3 matrix A by cyclic Jacobi rotations (Golub and Van Loan, Sec. 8.5):
 * A = V diag(ev) V^T, V orthonormal with det V = +1.  A is overwritten.
 */
static void sym_eig3(double A[3][3], double ev[3], double V[3][3])
{
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double nrm = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2] + 2.0 * off;
        if (off <= 1e-34 * nrm) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* the rotation in the (p, q) plane that zeroes A[p][q] */
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) {   /* A <- A G */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {   /* A <- G^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {   /* V <- V G */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) ev[i] = A[i][i];
    double d = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
               V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (d < 0) for (int i = 0; i < 3; ++i) V[i][2] = -V[i][2];
}

/*
 * I1 = tr(S) of the polar decomposition F = R S (Sec. 3.1), for det F > 0: F^T F = V Sigma^2 V^T, U = F V Sigma^-1,
 * R = U V^T, I1 = sum sigma_i.  g1 = vec(R).  H1 = sum_i lambda_i q_i q_i^T over the three twist modes
 * q_i = vec(U T_i V^T) / sqrt(2) (T_i the skew generator about axis i) with lambda_i = 2 / (sigma_j + sigma_k),
 * (i, j, k) cyclic: the second derivative of tr(S) is zero along the stretches and flips, and dR[dF] rotates with
 * the skew part of U^T dF V scaled by 1 / (sigma_j + sigma_k).
 */
static void polar_terms(tet_terms *T)
{
    double C[3][3], sg2[3], V[3][3], U[3][3], sg[3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[a][b] = T->F[0][a] * T->F[0][b] + T->F[1][a] * T->F[1][b] + T->F[2][a] * T->F[2][b];
    sym_eig3(C, sg2, V);
    for (int i = 0; i < 3; ++i) sg[i] = sqrt(sg2[i] > 0 ? sg2[i] : 0.0);
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 3; ++i)
            U[a][i] = (T->F[a][0] * V[0][i] + T->F[a][1] * V[1][i] + T->F[a][2] * V[2][i]) / sg[i];
    T->I1 = sg[0] + sg[1] + sg[2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            T->g1[3 * b + a] = U[a][0] * V[b][0] + U[a][1] * V[b][1] + U[a][2] * V[b][2];   /* R_ab, vec column-wise */
    memset(T->H1, 0, sizeof T->H1);
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        double lam = 2.0 / (sg[j] + sg[k]);
        /* T_i has +1 at (j, k) and -1 at (k, j): q = vec(U T_i V^T) / sqrt(2), (U T_i V^T)_ab = U_aj V_bk - U_ak V_bj */
        double q[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) q[3 * b + a] = (U[a][j] * V[b][k] - U[a][k] * V[b][j]) / sqrt(2.0);
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c < 9; ++c) T->H1[r][c] += lam * q[r] * q[c];
    }
}

static int tet_eval(const or_model *m, int32_t e, const double *x, tet_terms *T)
{
    const int32_t *v = m->tet + 4 * (size_t)e;
    const double (*Di)[3] = (const double (*)[3])(m->Dminv + 9 * (size_t)e);
    double Ds[3][3];
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a) Ds[a][c] = x[3 * (size_t)v[c + 1] + a] - x[3 * (size_t)v[0] + a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T->F[a][b] = Ds[a][0] * Di[0][b] + Ds[a][1] * Di[1][b] + Ds[a][2] * Di[2][b];
    double w[4][3];
    for (int b = 0; b < 3; ++b) {
        w[0][b] = -(Di[0][b] + Di[1][b] + Di[2][b]);
        for (int i = 1; i < 4; ++i) w[i][b] = Di[i - 1][b];
    }
    memset(T->J, 0, sizeof T->J);
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < 4; ++i) T->J[3 * b + a][3 * i + a] = w[i][b];
    double f[3][3];  /* columns of F */
    for (int b = 0; b < 3; ++b) for (int a = 0; a < 3; ++a) f[b][a] = T->F[a][b];
    double c0[3], c1[3], c2[3];
    cross3(f[1], f[2], c0);
    cross3(f[2], f[0], c1);
    cross3(f[0], f[1], c2);
    T->I2 = 0.0;
    for (int b = 0; b < 3; ++b) T->I2 += dot3(f[b], f[b]);
    T->I3 = dot3(f[0], c0);
    for (int b = 0; b < 3; ++b) for (int a = 0; a < 3; ++a) T->g2[3 * b + a] = 2.0 * f[b][a];
    for (int a = 0; a < 3; ++a) { T->g3[a] = c0[a]; T->g3[3 + a] = c1[a]; T->g3[6 + a] = c2[a]; }
    /* H3 = [[0, -^f2, ^f1], [^f2, 0, -^f0], [-^f1, ^f0, 0]] with ^f the cross-product matrix of f */
    memset(T->H3, 0, sizeof T->H3);
    const int blk[3][3] = {{-1, 2, 1}, {2, -1, 0}, {1, 0, -1}};   /* which column of F sits in block (r, c) */
    const double sg[3][3] = {{0, -1, 1}, {1, 0, -1}, {-1, 1, 0}};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            if (r == c) continue;
            const double *u = f[blk[r][c]];
            double hat[3][3] = {{0, -u[2], u[1]}, {u[2], 0, -u[0]}, {-u[1], u[0], 0}};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) T->H3[3 * r + i][3 * c + j] = sg[r][c] * hat[i][j];
        }
    if (!(T->I3 > 0.0)) return OR_ERR_INVERTED;
    double mu = m->mu[e], lam = m->lam[e];
    T->logI3 = log(T->I3);
    T->I1 = 3.0;
    memset(T->g1, 0, sizeof T->g1);
    memset(T->H1, 0, sizeof T->H1);
    T->Psi1 = T->Psi11 = T->Psi22 = 0.0;
    switch (m->p.model) {
    case OR_SNH:
        T->Psi2 = mu / 2.0;
        T->Psi3 = -mu + lam * (T->I3 - 1.0);
        T->Psi33 = lam;
        break;
    case OR_FCR:
    case OR_ARAP:
        polar_terms(T);
        T->Psi1 = -2.0 * mu;
        T->Psi2 = mu;
        T->Psi3 = m->p.model == OR_FCR ? lam * (T->I3 - 1.0) : 0.0;
        T->Psi33 = m->p.model == OR_FCR ? lam : 0.0;
        break;
    default:   /* OR_NH */
        T->Psi2 = mu / 2.0;
        T->Psi3 = (lam * T->logI3 - mu) / T->I3;
        T->Psi33 = (mu + lam * (1.0 - T->logI3)) / (T->I3 * T->I3);
    }
    T->scale = m->p.h * m->p.h * m->vol[e];
    return OR_OK;
}

/* the energy density of the model at the tet's invariants */
static double tet_psi(const or_model *m, int32_t e, const tet_terms *T)
{
    double mu = m->mu[e], lam = m->lam[e];
    switch (m->p.model) {
    case OR_SNH: return mu / 2.0 * (T->I2 - 3.0) - mu * (T->I3 - 1.0) + lam / 2.0 * (T->I3 - 1.0) * (T->I3 - 1.0);
    case OR_FCR: return mu * (T->I2 - 2.0 * T->I1 + 3.0) + lam / 2.0 * (T->I3 - 1.0) * (T->I3 - 1.0);
    case OR_ARAP: return mu * (T->I2 - 2.0 * T->I1 + 3.0);
    default: return mu / 2.0 * (T->I2 - 3.0) - mu * T->logI3 + lam / 2.0 * T->logI3 * T->logI3;
    }
}

/* ------------------------------------------------------------------------------------------------ energy, gradient, diag, pHp */

static int plane_d(const or_model *m, const double *xv, double *d)
{
    *d = dot3(m->plane_n, xv) - m->p.plane_o;
    return *d > 0.0 ? OR_OK : OR_ERR_PENETRATION;
}

/* E(x) (Eq. E) with the exact active set.  parts = {inertia, h^2 Psi, kappa sum b (pairs), kappa sum b (plane)} */
int or_energy(const or_model *m, const double *x, const double *xtilde, double *E_out, double *parts)
{
    int32_t nv = m->p.nv;
    double Ein = 0.0, Eel = 0.0, Ebp = 0.0, Ebl = 0.0;
    for (int32_t i = 0; i < nv; ++i) {
        double d[3];
        sub3(x + 3 * (size_t)i, xtilde + 3 * (size_t)i, d);
        Ein += 0.5 * m->mass[i] * dot3(d, d);
    }
    for (int32_t e = 0; e < m->p.nt; ++e) {
        tet_terms T;
        int st = tet_eval(m, e, x, &T);
        if (st) { set_err("inverted tet"); return st; }
        Eel += T.scale * tet_psi(m, e, &T);
    }
    pair_list L = {0};
    int st = find_pairs(m, x, m->p.dhat, 1, 0, &L);
    if (st) { free(L.v); return st; }
    for (int32_t k = 0; k < L.n; ++k) {
        if (!(L.v[k].d > 0.0)) { free(L.v); set_err("zero distance"); return OR_ERR_PENETRATION; }
        double bb[3];
        or_barrier_fn(L.v[k].d, m->p.dhat, bb);
        Ebp += m->p.kappa * bb[0];
    }
    free(L.v);
    if (m->p.has_plane)
        for (int32_t i = 0; i < nv; ++i) {
            double d;
            if (plane_d(m, x + 3 * (size_t)i, &d)) { set_err("vertex below plane"); return OR_ERR_PENETRATION; }
            double bb[3];
            or_barrier_fn(d, m->p.dhat, bb);
            Ebl += m->p.kappa * bb[0];
        }
    if (parts) { parts[0] = Ein; parts[1] = Eel; parts[2] = Ebp; parts[3] = Ebl; }
    *E_out = Ein + Eel + Ebp + Ebl;
    return isfinite(*E_out) ? OR_OK : OR_ERR_NONFINITE;
}

/*
 * Gradient g and Jacobi diagonal diag(H) of E at x (Eqs. E, Hessian), unmasked (kinematic vertices included).
 *   inertia:  g += M (x - xt), diag += m
 *   elastic:  g += h^2 V J^T (Psi2 g2 + Psi3 g3);  diag += h^2 V sum_i (Psi_ii diag(h_i) + Psi_i diag(h_{i+3}))
 *             with h_i = J^T g_i g_i^T J and h_{i+3} = J^T H_i J (the I1 terms vanish for NH and SNH)
 *   barrier:  g += kappa b'/d (dt/dx) t  (Eq. 8);  diag from Eqs. 9-11
 *   n_active receives the number of active pairs (NULL allowed).
 * With absmode set, every contribution to a vertex is added by the Euclidean length of its 3-vector instead (the
 * scale a rounding error of that vector is relative to, whatever the coordinate axes; the per-entry scale of the
 * parity tests), to all three entries: g receives m |x - xt| plus, per tet, h^2 V |dPsi/dF|_F |w_i| (the stress
 * taken as a whole; w_i the vertex's row of dF/dx) plus kappa |b'/d| |c_i| |t| per pair and kappa |b'| per plane
 * contact; diag receives m plus, per tet, the magnitudes of the six terms with each Jg_k entry replaced by the length
 * of the vertex's 3-vector Jg_k, plus kappa (|b''/d^2 - b'/d^3| c_i^2 |t|^2 + |b'/d| c_i^2) per pair and
 * kappa |b''| per plane contact.
 */
static int grad_diag_impl(const or_model *m, const double *x, const double *xtilde, double *g, double *diag,
                          int32_t *n_active, int absmode)
{
#define ACC(t) (absmode ? fabs(t) : (t))
    int32_t nv = m->p.nv;
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            if (absmode) {
                double dx[3];
                sub3(x + 3 * (size_t)i, xtilde + 3 * (size_t)i, dx);
                g[3 * (size_t)i + a] = m->mass[i] * sqrt(dot3(dx, dx));
            } else {
                g[3 * (size_t)i + a] = m->mass[i] * (x[3 * (size_t)i + a] - xtilde[3 * (size_t)i + a]);
            }
            diag[3 * (size_t)i + a] = m->mass[i];
        }
    for (int32_t e = 0; e < m->p.nt; ++e) {
        tet_terms T;
        int st = tet_eval(m, e, x, &T);
        if (st) { set_err("inverted tet"); return st; }
        const int32_t *v = m->tet + 4 * (size_t)e;
        double dPsi[9];
        for (int r = 0; r < 9; ++r) dPsi[r] = T.Psi1 * T.g1[r] + T.Psi2 * T.g2[r] + T.Psi3 * T.g3[r];
        double Jg1[12], Jg2[12], Jg3[12], dg[12], dh[12];
        for (int q = 0; q < 12; ++q) {
            double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            for (int r = 0; r < 9; ++r) {
                s0 += T.J[r][q] * dPsi[r]; s1 += T.J[r][q] * T.g1[r];
                s2 += T.J[r][q] * T.g2[r]; s3 += T.J[r][q] * T.g3[r];
            }
            dg[q] = s0; Jg1[q] = s1; Jg2[q] = s2; Jg3[q] = s3;
        }
        if (absmode) {   /* Euclidean lengths of the vertex's 3-vectors: dPsi w_i and J g_k restricted to vertex i */
            double nP = 0.0;
            for (int r = 0; r < 9; ++r) nP += dPsi[r] * dPsi[r];
            nP = sqrt(nP);
            for (int i = 0; i < 4; ++i) {
                double nw = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0;
                for (int b = 0; b < 3; ++b) nw += T.J[3 * b][3 * i] * T.J[3 * b][3 * i];
                for (int a = 0; a < 3; ++a) {
                    const int q = 3 * i + a;
                    n1 += Jg1[q] * Jg1[q]; n2 += Jg2[q] * Jg2[q]; n3 += Jg3[q] * Jg3[q];
                }
                for (int a = 0; a < 3; ++a) {
                    dg[3 * i + a] = nP * sqrt(nw);
                    Jg1[3 * i + a] = sqrt(n1); Jg2[3 * i + a] = sqrt(n2); Jg3[3 * i + a] = sqrt(n3);
                }
            }
        }
        /* diag(J^T H J) for H1, H2 = 2 I and H3 */
        for (int q = 0; q < 12; ++q) {
            double h4 = 0, h5 = 0, h6 = 0;
            for (int r = 0; r < 9; ++r) {
                h5 += T.J[r][q] * 2.0 * T.J[r][q];
                double HJ = 0, H1J = 0;
                for (int s = 0; s < 9; ++s) { HJ += T.H3[r][s] * T.J[s][q]; H1J += T.H1[r][s] * T.J[s][q]; }
                h6 += T.J[r][q] * HJ;
                h4 += T.J[r][q] * H1J;
            }
            dh[q] = ACC(T.Psi11 * Jg1[q] * Jg1[q]) + ACC(T.Psi22 * Jg2[q] * Jg2[q]) + ACC(T.Psi33 * Jg3[q] * Jg3[q]) +
                    ACC(T.Psi1 * h4) + ACC(T.Psi2 * h5) + ACC(T.Psi3 * h6);
        }
        for (int i = 0; i < 4; ++i)
            for (int a = 0; a < 3; ++a) {
                g[3 * (size_t)v[i] + a] += T.scale * dg[3 * i + a];
                diag[3 * (size_t)v[i] + a] += T.scale * dh[3 * i + a];
            }
    }
    pair_list L = {0};
    int st = find_pairs(m, x, m->p.dhat, 1, 0, &L);
    if (st) { free(L.v); return st; }
    double kap = m->p.kappa, dh_ = m->p.dhat;
    for (int32_t k = 0; k < L.n; ++k) {
        const or_pair *P = &L.v[k];
        double d = P->d;
        if (!(d > 0.0)) { free(L.v); set_err("zero distance"); return OR_ERR_PENETRATION; }
        double bb[3];
        or_barrier_fn(d, dh_, bb);
        double coef_tt = kap * (bb[2] / (d * d) - bb[1] / (d * d * d));  /* multiplies (dt/dx t)(dt/dx t)^T */
        double coef_I = kap * bb[1] / d;                                 /* multiplies (dt/dx)(dt/dx)^T */
        const double tn = sqrt(dot3(P->t, P->t));
        for (int i = 0; i < 4; ++i)
            for (int a = 0; a < 3; ++a) {
                double ct = P->c[i] * P->t[a];
                if (absmode) {
                    const double ctn = fabs(P->c[i]) * tn;
                    g[3 * (size_t)P->v[i] + a] += fabs(coef_I) * ctn;
                    diag[3 * (size_t)P->v[i] + a] += fabs(coef_tt) * ctn * ctn + fabs(coef_I) * P->c[i] * P->c[i];
                } else {
                    g[3 * (size_t)P->v[i] + a] += coef_I * ct;
                    diag[3 * (size_t)P->v[i] + a] += coef_tt * ct * ct + coef_I * P->c[i] * P->c[i];
                }
            }
    }
    if (n_active) *n_active = L.n;
    free(L.v);
    if (m->p.has_plane)
        for (int32_t i = 0; i < nv; ++i) {
            double d;
            if (plane_d(m, x + 3 * (size_t)i, &d)) { set_err("vertex below plane"); return OR_ERR_PENETRATION; }
            if (!(d < dh_)) continue;
            double bb[3];
            or_barrier_fn(d, dh_, bb);
            for (int a = 0; a < 3; ++a) {
                if (absmode) {
                    g[3 * (size_t)i + a] += fabs(kap * bb[1]) * sqrt(dot3(m->plane_n, m->plane_n));
                    diag[3 * (size_t)i + a] += fabs(kap * bb[2]) * dot3(m->plane_n, m->plane_n);
                } else {
                    g[3 * (size_t)i + a] += kap * bb[1] * m->plane_n[a];
                    diag[3 * (size_t)i + a] += kap * bb[2] * m->plane_n[a] * m->plane_n[a];
                }
            }
        }
    for (size_t q = 0; q < 3 * (size_t)nv; ++q)
        if (!isfinite(g[q]) || !isfinite(diag[q])) { set_err("non-finite gradient"); return OR_ERR_NONFINITE; }
    return OR_OK;
#undef ACC
}

int or_grad_diag(const or_model *m, const double *x, const double *xtilde, double *g, double *diag, int32_t *n_active)
{
    return grad_diag_impl(m, x, xtilde, g, diag, n_active, 0);
}

/* Per-entry magnitude sums of the contributions to g and diag(H) at x (grad_diag_impl's absmode). */
int or_grad_diag_scale(const or_model *m, const double *x, const double *xtilde, double *gs, double *ds)
{
    return grad_diag_impl(m, x, xtilde, gs, ds, NULL, 1);
}

/*
 * p^T H p at x (Eq. Hessian): p^T M p + h^2 sum_e V_e sum_i (Psi_ii p^T h_i p + Psi_i p^T h_{i+3} p)
 * + kappa sum_C [(b''/d^2 - b'/d^3)(p^T dt/dx t)^2 + b'/d ||p^T dt/dx||^2]   (Eqs. 12, 13; frozen c)
 */
int or_pHp(const or_model *m, const double *x, const double *p, double *out)
{
    int32_t nv = m->p.nv;
    double s = 0.0;
    for (int32_t i = 0; i < nv; ++i) s += m->mass[i] * dot3(p + 3 * (size_t)i, p + 3 * (size_t)i);
    for (int32_t e = 0; e < m->p.nt; ++e) {
        tet_terms T;
        int st = tet_eval(m, e, x, &T);
        if (st) { set_err("inverted tet"); return st; }
        const int32_t *v = m->tet + 4 * (size_t)e;
        double pe[12], Jp[9];
        for (int i = 0; i < 4; ++i) for (int a = 0; a < 3; ++a) pe[3 * i + a] = p[3 * (size_t)v[i] + a];
        for (int r = 0; r < 9; ++r) { double acc = 0; for (int q = 0; q < 12; ++q) acc += T.J[r][q] * pe[q]; Jp[r] = acc; }
        double g1Jp = 0, g2Jp = 0, g3Jp = 0, h4 = 0, h5 = 0, h6 = 0;
        for (int r = 0; r < 9; ++r) {
            g1Jp += T.g1[r] * Jp[r];
            g2Jp += T.g2[r] * Jp[r];
            g3Jp += T.g3[r] * Jp[r];
            h5 += Jp[r] * 2.0 * Jp[r];
            double HJp = 0, H1Jp = 0;
            for (int q = 0; q < 9; ++q) { HJp += T.H3[r][q] * Jp[q]; H1Jp += T.H1[r][q] * Jp[q]; }
            h6 += Jp[r] * HJp;
            h4 += Jp[r] * H1Jp;
        }
        s += T.scale * (T.Psi11 * g1Jp * g1Jp + T.Psi22 * g2Jp * g2Jp + T.Psi33 * g3Jp * g3Jp + T.Psi1 * h4 +
                        T.Psi2 * h5 + T.Psi3 * h6);
    }
    pair_list L = {0};
    int st = find_pairs(m, x, m->p.dhat, 1, 0, &L);
    if (st) { free(L.v); return st; }
    double kap = m->p.kappa, dh_ = m->p.dhat;
    for (int32_t k = 0; k < L.n; ++k) {
        const or_pair *P = &L.v[k];
        double d = P->d;
        if (!(d > 0.0)) { free(L.v); set_err("zero distance"); return OR_ERR_PENETRATION; }
        double bb[3];
        or_barrier_fn(d, dh_, bb);
        double cp[3] = {0, 0, 0};   /* p^T dt/dx = sum_i c_i p_i */
        for (int i = 0; i < 4; ++i) for (int a = 0; a < 3; ++a) cp[a] += P->c[i] * p[3 * (size_t)P->v[i] + a];
        double cpt = dot3(cp, P->t);
        s += kap * ((bb[2] / (d * d) - bb[1] / (d * d * d)) * cpt * cpt + bb[1] / d * dot3(cp, cp));
    }
    free(L.v);
    if (m->p.has_plane)
        for (int32_t i = 0; i < nv; ++i) {
            double d;
            if (plane_d(m, x + 3 * (size_t)i, &d)) { set_err("vertex below plane"); return OR_ERR_PENETRATION; }
            if (!(d < dh_)) continue;
            double bb[3];
            or_barrier_fn(d, dh_, bb);
            double np = dot3(m->plane_n, p + 3 * (size_t)i);
            s += kap * bb[2] * np * np;
        }
    *out = s;
    return isfinite(s) ? OR_OK : OR_ERR_NONFINITE;
}

/*
 * Active pairs at x: rows of out_idx are (type, v0, v1, v2, v3), out_d their distances.  threshold <= 0 means
 * dhat.  brute = 1 tests all pairs.  Returns the count through *count (may exceed max; only max rows written).
 */
int or_active_pairs(const or_model *m, const double *x, int32_t brute, double threshold, int32_t use_excl,
                    int32_t *out_idx, double *out_d, double *out_c, int32_t max, int32_t *count)
{
    pair_list L = {0};
    int st = find_pairs(m, x, threshold > 0 ? threshold : m->p.dhat, use_excl, brute, &L);
    if (st) { free(L.v); return st; }
    for (int32_t k = 0; k < L.n && k < max; ++k) {
        out_idx[5 * (size_t)k] = L.v[k].type;
        for (int i = 0; i < 4; ++i) out_idx[5 * (size_t)k + 1 + i] = L.v[k].v[i];
        if (out_d) out_d[k] = L.v[k].d;
        if (out_c) memcpy(out_c + 4 * (size_t)k, L.v[k].c, 4 * sizeof(double));
    }
    *count = L.n;
    free(L.v);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------------ PNCG (Sec. 4, Algorithm 1) */

/*
 * Search direction (Sec. 4.1-4.2).  n = vector length.  p holds p_k on entry and p_{k+1} on return.
 * k == 0: beta = 0.  rule 0 (PR+): beta = max(0, g1^T P1 (g1 - g0) / (g0^T P0 g0)).
 * rule 1 (DK, preconditioned): beta = g1^T P1 y / (y^T p) - (y^T P1 y / y^T p) (p^T g1 / y^T p), y = g1 - g0.
 * p_{k+1} = -P1 g1 + beta p_k; if g1^T p_{k+1} >= 0 the direction restarts with beta = 0.
 */
int or_ncg_direction(int32_t n, const double *g1, const double *P1, const double *g0, const double *P0, double *p,
                     int32_t k, int32_t rule, double *beta_out, double *gp_out, int32_t *restarted)
{
    double beta = 0.0;
    if (k > 0) {
        if (rule == 0) {
            double num = 0.0, den = 0.0;
            for (int32_t i = 0; i < n; ++i) {
                num += g1[i] * P1[i] * (g1[i] - g0[i]);
                den += g0[i] * P0[i] * g0[i];
            }
            beta = den > 0.0 ? num / den : 0.0;
            if (beta < 0.0) beta = 0.0;
        } else {
            double gPy = 0.0, yPy = 0.0, yp = 0.0, pg = 0.0;
            for (int32_t i = 0; i < n; ++i) {
                double y = g1[i] - g0[i];
                gPy += g1[i] * P1[i] * y;
                yPy += y * P1[i] * y;
                yp += y * p[i];
                pg += p[i] * g1[i];
            }
            beta = fabs(yp) < 1e-30 ? 0.0 : gPy / yp - (yPy / yp) * (pg / yp);
        }
    }
    double gp = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        p[i] = -P1[i] * g1[i] + beta * p[i];
        gp += g1[i] * p[i];
    }
    *restarted = 0;
    if (gp >= 0.0 && beta != 0.0) {
        beta = 0.0;
        gp = 0.0;
        for (int32_t i = 0; i < n; ++i) { p[i] = -P1[i] * g1[i]; gp += g1[i] * p[i]; }
        *restarted = 1;
    }
    *beta_out = beta;
    *gp_out = gp;
    return OR_OK;
}

/* largest per-vertex Euclidean length (pnorm 0) or largest absolute component (pnorm 1) of p [nv][3] */
double or_pmax(int32_t nv, const double *p, int32_t pnorm)
{
    double mx = 0.0;
    for (int32_t i = 0; i < nv; ++i) {
        double v;
        if (pnorm == 0) v = sqrt(dot3(p + 3 * (size_t)i, p + 3 * (size_t)i));
        else { v = fabs(p[3 * (size_t)i]); if (fabs(p[3 * (size_t)i + 1]) > v) v = fabs(p[3 * (size_t)i + 1]); if (fabs(p[3 * (size_t)i + 2]) > v) v = fabs(p[3 * (size_t)i + 2]); }
        if (v > mx) mx = v;
    }
    return mx;
}

/*
 * Step size (Sec. 4.3, Eqs. linesearch, upper, alpha) and the predicted decrease (Sec. 4.4):
 * alpha_bar = -g^T p / p^T H p, alpha_upper = dhat / (2 pmax), alpha = min of the two;
 * alpha = alpha_upper when p^T H p <= 0 or alpha_bar is not finite; alpha = 0 when pmax = 0.
 * out = {alpha, alpha_bar, alpha_upper, dE, capped}
 */
void or_ncg_alpha(double gp, double pHp, double pmax, double dhat, double *out)
{
    double au = pmax > 0.0 ? dhat / (2.0 * pmax) : 0.0;
    double ab = -gp / pHp;
    double a;
    int capped;
    if (!(pHp > 0.0) || !isfinite(ab)) { a = au; capped = 1; }
    else if (ab < au) { a = ab; capped = 0; }
    else { a = au; capped = 1; }
    out[0] = a; out[1] = ab; out[2] = au;
    out[3] = -a * gp - 0.5 * a * a * pHp;
    out[4] = capped;
}

/* smallest diagonal entry, as a fraction of the vertex mass, that the Jacobi preconditioner inverts */
#define OR_JACOBI_FLOOR 1e-3

/* Jacobi preconditioner P = diag(H)^-1 (Sec. 4.2) where diag > 1e-3 m_v, else 1 / m_v; kinematic vertices get
   g = 0 and P = 0 */
static void jacobi(const or_model *m, double *g1, const double *d1, double *P1)
{
    for (int32_t i = 0; i < m->p.nv; ++i)
        for (int a = 0; a < 3; ++a) {
            size_t q = 3 * (size_t)i + a;
            if (m->fixed[i]) { g1[q] = 0.0; P1[q] = 0.0; continue; }
            P1[q] = d1[q] > OR_JACOBI_FLOOR * m->mass[i] ? 1.0 / d1[q] : 1.0 / m->mass[i];
        }
}

/* vertices within dhat of the plane (reported, like the pair count) */
static int32_t count_plane(const or_model *m, const double *x)
{
    int32_t nplane = 0;
    if (m->p.has_plane)
        for (int32_t i = 0; i < m->p.nv; ++i) if (dot3(m->plane_n, x + 3 * (size_t)i) - m->p.plane_o < m->p.dhat) ++nplane;
    return nplane;
}

/*
 * One iteration of Algorithm 1 at x = x_k.  In: g = g_k, P = P_k, p = p_k (ignored at k = 0).
 * Out: x = x_{k+1}, g = g_{k+1} (at x_k, kinematic entries zero), P = P_{k+1}, p = p_{k+1}; scalars in *s.
 */
int or_iteration(const or_model *m, double *x, const double *xtilde, double *g, double *P, double *p, or_ncg_scalars *s)
{
    int32_t nv = m->p.nv;
    size_t n = 3 * (size_t)nv;
    double *g1 = malloc(sizeof(double) * n), *d1 = malloc(sizeof(double) * n), *P1 = malloc(sizeof(double) * n);
    if (!g1 || !d1 || !P1) { free(g1); free(d1); free(P1); return OR_ERR_OOM; }
    int32_t nact = 0;
    int st = or_grad_diag(m, x, xtilde, g1, d1, &nact);   /* C <- ComputeConstraintSet; g, diag */
    if (st) { free(g1); free(d1); free(P1); return st; }
    jacobi(m, g1, d1, P1);
    int32_t nplane = count_plane(m, x);
    double beta, gp;
    int32_t rs;
    or_ncg_direction((int32_t)n, g1, P1, g, P, p, s->k, m->p.beta_rule, &beta, &gp, &rs);
    double pmax = or_pmax(nv, p, m->p.pnorm);
    double pHp;
    st = or_pHp(m, x, p, &pHp);
    if (st) { free(g1); free(d1); free(P1); return st; }
    double al[5];
    or_ncg_alpha(gp, pHp, pmax, m->p.dhat, al);
    for (size_t q = 0; q < n; ++q) x[q] += al[0] * p[q];
    memcpy(g, g1, sizeof(double) * n);
    memcpy(P, P1, sizeof(double) * n);
    free(g1); free(d1); free(P1);
    s->beta = beta; s->gp = gp; s->pHp = pHp; s->pmax = pmax;
    s->alpha = al[0]; s->alpha_bar = al[1]; s->alpha_up = al[2]; s->dE = al[3]; s->capped = (int32_t)al[4];
    s->restarted = rs; s->n_active = nact; s->n_plane = nplane;
    if (s->k == 0) s->dE0 = s->dE;
    s->k += 1;
    return OR_OK;
}

/*
 * One iteration with splitting (Sec. 5.2) over ngroups vertex groups, group[i] in 0 .. ngroups-1 for vertex i (a
 * group need not be contiguous: an object, or the collision or non-collision part of one).  Gradient and
 * preconditioner are those of the whole scene (pairs between groups included).  Each group then takes its own beta
 * and direction over its own entries (in vertex order; Sec. 4.1-4.2), its own max |p_v|, and its own step along
 * p_G, which is p with every other group's entries zero: alpha_G = min(dhat / (2 max |p_v|), -g^T p_G / p_G^T H p_G)
 * (Sec. 4.3), i.e. the step of the quadratic model of E along p_G with the other groups held still.  All p_G^T H p_G
 * are taken at x_k before any group moves.  moving (nullable): groups with moving[G] = 0 (converged under the eps
 * rule) keep their direction but take no step.  s: ngroups scalars, each with its own k and dE0.
 */
int or_iteration_groups(const or_model *m, int32_t ngroups, const int32_t *group, const int32_t *moving, double *x,
                        const double *xtilde, double *g, double *P, double *p, or_ncg_scalars *s)
{
    int32_t nv = m->p.nv;
    size_t n = 3 * (size_t)nv;
    if (ngroups < 1) { set_err("at least one group"); return OR_ERR_ARG; }
    for (int32_t i = 0; i < nv; ++i)
        if (group[i] < 0 || group[i] >= ngroups) { set_err("group label out of range"); return OR_ERR_ARG; }
    double *g1 = malloc(sizeof(double) * n), *d1 = malloc(sizeof(double) * n), *P1 = malloc(sizeof(double) * n);
    double *po = calloc(n, sizeof(double)), *al = malloc(sizeof(double) * 5 * (size_t)ngroups);
    double *t = malloc(sizeof(double) * 5 * n);   /* a group's entries gathered: g1, P1, g, P, p */
    int32_t *idx = malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    if (!g1 || !d1 || !P1 || !po || !al || !t || !idx) {
        free(g1); free(d1); free(P1); free(po); free(al); free(t); free(idx);
        return OR_ERR_OOM;
    }
    int32_t nact = 0;
    int st = or_grad_diag(m, x, xtilde, g1, d1, &nact);
    if (st) goto done;
    jacobi(m, g1, d1, P1);
    int32_t nplane = count_plane(m, x);
    for (int32_t G = 0; G < ngroups; ++G) {
        int32_t nq = 0;
        for (int32_t i = 0; i < nv; ++i) if (group[i] == G) idx[nq++] = i;
        double *tg1 = t, *tP1 = t + n, *tg = t + 2 * n, *tP = t + 3 * n, *tp = t + 4 * n;
        for (int32_t j = 0; j < nq; ++j)
            for (int a = 0; a < 3; ++a) {
                size_t q = 3 * (size_t)idx[j] + a, r = 3 * (size_t)j + a;
                tg1[r] = g1[q]; tP1[r] = P1[q]; tg[r] = g[q]; tP[r] = P[q]; tp[r] = p[q];
            }
        or_ncg_direction(3 * nq, tg1, tP1, tg, tP, tp, s[G].k, m->p.beta_rule, &s[G].beta, &s[G].gp, &s[G].restarted);
        s[G].pmax = or_pmax(nq, tp, m->p.pnorm);
        for (int32_t j = 0; j < nq; ++j)
            for (int a = 0; a < 3; ++a) p[3 * (size_t)idx[j] + a] = tp[3 * (size_t)j + a];
    }
    for (int32_t G = 0; G < ngroups; ++G) {
        for (int32_t i = 0; i < nv; ++i)
            for (int a = 0; a < 3; ++a) po[3 * (size_t)i + a] = group[i] == G ? p[3 * (size_t)i + a] : 0.0;
        st = or_pHp(m, x, po, &s[G].pHp);
        if (st) goto done;
        or_ncg_alpha(s[G].gp, s[G].pHp, s[G].pmax, m->p.dhat, al + 5 * (size_t)G);
    }
    for (int32_t G = 0; G < ngroups; ++G) {
        const double *a = al + 5 * (size_t)G;
        double step = (moving && !moving[G]) ? 0.0 : a[0];
        for (int32_t i = 0; i < nv; ++i)
            if (group[i] == G)
                for (int c = 0; c < 3; ++c) x[3 * (size_t)i + c] += step * p[3 * (size_t)i + c];
        s[G].alpha = step; s[G].alpha_bar = a[1]; s[G].alpha_up = a[2]; s[G].dE = a[3]; s[G].capped = (int32_t)a[4];
        s[G].n_active = nact; s[G].n_plane = nplane;
        if (s[G].k == 0) s[G].dE0 = s[G].dE;
        s[G].k += 1;
    }
    memcpy(g, g1, sizeof(double) * n);
    memcpy(P, P1, sizeof(double) * n);
done:
    free(g1); free(d1); free(P1); free(po); free(al); free(t); free(idx);
    return st;
}

/*
 * Per-object splitting (Sec. 5.2) with the objects as contiguous vertex ranges off[o] .. off[o+1]-1: the group
 * iteration above with group = object.
 */
int or_iteration_split(const or_model *m, int32_t nobj, const int32_t *off, const int32_t *moving, double *x,
                       const double *xtilde, double *g, double *P, double *p, or_ncg_scalars *s)
{
    int32_t nv = m->p.nv;
    if (nobj < 1 || off[0] != 0 || off[nobj] != nv) { set_err("object ranges must cover the vertices"); return OR_ERR_ARG; }
    for (int32_t o = 0; o < nobj; ++o)
        if (off[o + 1] < off[o]) { set_err("object ranges must be non-decreasing"); return OR_ERR_ARG; }
    int32_t *group = malloc(sizeof(int32_t) * (size_t)nv);
    if (!group) return OR_ERR_OOM;
    for (int32_t o = 0; o < nobj; ++o)
        for (int32_t i = off[o]; i < off[o + 1]; ++i) group[i] = o;
    int st = or_iteration_groups(m, nobj, group, moving, x, xtilde, g, P, p, s);
    free(group);
    return st;
}

/*
 * The vertices in contact at x: mark[i] = 1 for every vertex of a pair of the active set (d < dhat, rest-pose
 * exclusions applied) and every vertex within dhat of the plane, else 0.  The collision part of an object for
 * the split of Sec. 5.2.
 */
int or_contact_vertices(const or_model *m, const double *x, int32_t *mark)
{
    for (int32_t i = 0; i < m->p.nv; ++i) mark[i] = 0;
    pair_list L = {0};
    int st = find_pairs(m, x, m->p.dhat, 1, 0, &L);
    if (st) { free(L.v); return st; }
    for (int32_t k = 0; k < L.n; ++k)
        for (int i = 0; i < 4; ++i) mark[L.v[k].v[i]] = 1;
    free(L.v);
    if (m->p.has_plane)
        for (int32_t i = 0; i < m->p.nv; ++i)
            if (dot3(m->plane_n, x + 3 * (size_t)i) - m->p.plane_o < m->p.dhat) mark[i] = 1;
    return OR_OK;
}

/*
 * One time step (Algorithm 1 with the implicit-Euler prediction of Sec. 3):
 *   xt = x^t + h v^t + h^2 gravity (free vertices); kinematic vertices jump to their targets
 *   (targets [n_fixed][3] in increasing vertex order, NULL = stay);  x_0 = x^t with those targets;
 *   iterate until iters or, when eps > 0, until Delta E < eps Delta E_0;  v = (x - x^t) / h.
 * trace (NULL allowed) receives per iteration {beta, gp, pHp, pmax, alpha, dE, n_active, capped}.
 */
int or_step(const or_model *m, double *x, double *v, const double *targets, int32_t iters, double eps, double *trace,
            int32_t *iters_done)
{
    int32_t nv = m->p.nv;
    size_t n = 3 * (size_t)nv;
    double h = m->p.h;
    double *xt = malloc(sizeof(double) * n), *xtil = malloc(sizeof(double) * n);
    double *g = calloc(n, sizeof(double)), *P = calloc(n, sizeof(double)), *p = calloc(n, sizeof(double));
    if (!xt || !xtil || !g || !P || !p) { free(xt); free(xtil); free(g); free(P); free(p); return OR_ERR_OOM; }
    memcpy(xt, x, sizeof(double) * n);
    int32_t f = 0;
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) xtil[3 * (size_t)i + a] = x[3 * (size_t)i + a] + h * v[3 * (size_t)i + a] + h * h * m->p.gravity[a];
    for (int32_t i = 0; i < nv; ++i)
        if (m->fixed[i]) {
            for (int a = 0; a < 3; ++a) {
                double tg = targets ? targets[3 * (size_t)f + a] : x[3 * (size_t)i + a];
                x[3 * (size_t)i + a] = tg;
                xtil[3 * (size_t)i + a] = tg;
            }
            ++f;
        }
    or_ncg_scalars s;
    memset(&s, 0, sizeof s);
    int st = OR_OK;
    int32_t k;
    for (k = 0; k < iters; ++k) {
        st = or_iteration(m, x, xtil, g, P, p, &s);
        if (st) break;
        if (trace) {
            double *tr = trace + 8 * (size_t)k;
            tr[0] = s.beta; tr[1] = s.gp; tr[2] = s.pHp; tr[3] = s.pmax; tr[4] = s.alpha; tr[5] = s.dE;
            tr[6] = s.n_active; tr[7] = s.capped;
        }
        if (eps > 0.0 && s.dE < eps * s.dE0) { ++k; break; }
    }
    if (iters_done) *iters_done = k;
    if (st == OR_OK)
        for (size_t q = 0; q < n; ++q) v[q] = (x[q] - xt[q]) / h;
    free(xt); free(xtil); free(g); free(P); free(p);
    return st;
}

/* the prediction xt of a step (same arithmetic as or_step) for energy reporting */
void or_predict(const or_model *m, const double *x, const double *v, const double *targets, double *xtil)
{
    int32_t nv = m->p.nv, f = 0;
    double h = m->p.h;
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) xtil[3 * (size_t)i + a] = x[3 * (size_t)i + a] + h * v[3 * (size_t)i + a] + h * h * m->p.gravity[a];
    for (int32_t i = 0; i < nv; ++i)
        if (m->fixed[i]) {
            for (int a = 0; a < 3; ++a) xtil[3 * (size_t)i + a] = targets ? targets[3 * (size_t)f + a] : x[3 * (size_t)i + a];
            ++f;
        }
}

/* ------------------------------------------------------------------------------------------------ discrete collision check */

static double orient3(const double *a, const double *b, const double *c, const double *d)
{
    double u[3], v[3], w[3], cr[3];
    sub3(b, a, u); sub3(c, a, v); sub3(d, a, w);
    cross3(u, v, cr);
    return dot3(cr, w);
}

/*
 * Number of (surface edge, surface triangle) pairs that share no vertex and whose segment crosses the triangle
 * (strict orientation tests), plus vertices on or below the plane: the per-frame penetration check of Sec. 6.3.
 */
int32_t or_intersections(const or_model *m, const double *x)
{
    int32_t cnt = 0;
    for (int32_t e = 0; e < m->ne; ++e) {
        int32_t a = m->edge[2 * e], b = m->edge[2 * e + 1];
        const double *pa = x + 3 * (size_t)a, *pb = x + 3 * (size_t)b;
        for (int32_t f = 0; f < m->nf; ++f) {
            const int32_t *t = m->tri + 3 * (size_t)f;
            if (t[0] == a || t[1] == a || t[2] == a || t[0] == b || t[1] == b || t[2] == b) continue;
            const double *p0 = x + 3 * (size_t)t[0], *p1 = x + 3 * (size_t)t[1], *p2 = x + 3 * (size_t)t[2];
            double sa = orient3(p0, p1, p2, pa), sb = orient3(p0, p1, p2, pb);
            if (!((sa > 0 && sb < 0) || (sa < 0 && sb > 0))) continue;
            double s0 = orient3(pa, pb, p0, p1), s1 = orient3(pa, pb, p1, p2), s2 = orient3(pa, pb, p2, p0);
            if ((s0 > 0 && s1 > 0 && s2 > 0) || (s0 < 0 && s1 < 0 && s2 < 0)) ++cnt;
        }
    }
    if (m->p.has_plane)
        for (int32_t i = 0; i < m->p.nv; ++i)
            if (!(dot3(m->plane_n, x + 3 * (size_t)i) - m->p.plane_o > 0.0)) ++cnt;
    return cnt;
}

/* ------------------------------------------------------------------------------------------------ differentiation */

/*
 * H v at x, H the Hessian of E (Eq. Hessian) as p^T H p sees it: the lumped mass, the elastic six-term split of
 * Sec. 3.1 (sum_i Psi_ii g_i g_i^T + Psi_i H_i mapped by vec(dF/dx)), the barrier with the closest points frozen
 * (Eq. 9: (b''/d^2 - b'/d^3) (dt/dx t)(dt/dx t)^T + b'/d (dt/dx)(dt/dx)^T) and the plane barrier b'' n n^T.  Rows
 * and columns of kinematic vertices are dropped (their entries of v are ignored, of out set to zero).  The paper
 * has no adjoint: this is the vector form of or_pHp (v^T H v equals it), for the oracle's own adjoint step.
 */
int or_hvp(const or_model *m, const double *x, const double *v_in, double *out)
{
    int32_t nv = m->p.nv;
    size_t n = 3 * (size_t)nv;
    double *v = malloc(sizeof(double) * n);
    if (!v) return OR_ERR_OOM;
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) v[3 * (size_t)i + a] = m->fixed[i] ? 0.0 : v_in[3 * (size_t)i + a];
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) out[3 * (size_t)i + a] = m->mass[i] * v[3 * (size_t)i + a];
    for (int32_t e = 0; e < m->p.nt; ++e) {
        tet_terms T;
        int st = tet_eval(m, e, x, &T);
        if (st) { free(v); set_err("inverted tet"); return st; }
        const int32_t *vi = m->tet + 4 * (size_t)e;
        double ve[12], Jv[9], HJv[9];
        for (int i = 0; i < 4; ++i) for (int a = 0; a < 3; ++a) ve[3 * i + a] = v[3 * (size_t)vi[i] + a];
        for (int r = 0; r < 9; ++r) { double acc = 0; for (int q = 0; q < 12; ++q) acc += T.J[r][q] * ve[q]; Jv[r] = acc; }
        double g1Jv = 0, g2Jv = 0, g3Jv = 0;
        for (int r = 0; r < 9; ++r) { g1Jv += T.g1[r] * Jv[r]; g2Jv += T.g2[r] * Jv[r]; g3Jv += T.g3[r] * Jv[r]; }
        for (int r = 0; r < 9; ++r) {
            double H1 = 0, H3 = 0;
            for (int q = 0; q < 9; ++q) { H1 += T.H1[r][q] * Jv[q]; H3 += T.H3[r][q] * Jv[q]; }
            HJv[r] = T.Psi11 * g1Jv * T.g1[r] + T.Psi22 * g2Jv * T.g2[r] + T.Psi33 * g3Jv * T.g3[r] + T.Psi1 * H1 +
                     T.Psi2 * 2.0 * Jv[r] + T.Psi3 * H3;
        }
        for (int q = 0; q < 12; ++q) {
            double acc = 0;
            for (int r = 0; r < 9; ++r) acc += T.J[r][q] * HJv[r];
            out[3 * (size_t)vi[q / 3] + q % 3] += T.scale * acc;
        }
    }
    pair_list L = {0};
    int st = find_pairs(m, x, m->p.dhat, 1, 0, &L);
    if (st) { free(L.v); free(v); return st; }
    double kap = m->p.kappa, dh_ = m->p.dhat;
    for (int32_t k = 0; k < L.n; ++k) {
        const or_pair *P = &L.v[k];
        double d = P->d;
        if (!(d > 0.0)) { free(L.v); free(v); set_err("zero distance"); return OR_ERR_PENETRATION; }
        double bb[3];
        or_barrier_fn(d, dh_, bb);
        double A = kap * (bb[2] / (d * d) - bb[1] / (d * d * d)), Bc = kap * bb[1] / d;
        double cv[3] = {0, 0, 0};   /* (dt/dx)^T v = sum_i c_i v_i */
        for (int i = 0; i < 4; ++i) for (int a = 0; a < 3; ++a) cv[a] += P->c[i] * v[3 * (size_t)P->v[i] + a];
        double cvt = dot3(cv, P->t);
        for (int i = 0; i < 4; ++i)
            for (int a = 0; a < 3; ++a) out[3 * (size_t)P->v[i] + a] += P->c[i] * (A * cvt * P->t[a] + Bc * cv[a]);
    }
    free(L.v);
    if (m->p.has_plane)
        for (int32_t i = 0; i < nv; ++i) {
            double d;
            if (plane_d(m, x + 3 * (size_t)i, &d)) { free(v); set_err("vertex below plane"); return OR_ERR_PENETRATION; }
            if (!(d < dh_)) continue;
            double bb[3];
            or_barrier_fn(d, dh_, bb);
            double nvv = dot3(m->plane_n, v + 3 * (size_t)i);
            for (int a = 0; a < 3; ++a) out[3 * (size_t)i + a] += kap * bb[2] * nvv * m->plane_n[a];
        }
    for (int32_t i = 0; i < nv; ++i)
        if (m->fixed[i]) for (int a = 0; a < 3; ++a) out[3 * (size_t)i + a] = 0.0;
    free(v);
    for (size_t q = 0; q < n; ++q) if (!isfinite(out[q])) { set_err("non-finite H v"); return OR_ERR_NONFINITE; }
    return OR_OK;
}

/*
 * The reverse of one time step x_t -> x_{t+1} = argmin E(x; x~_t), v_{t+1} = (x_{t+1} - x_t)/h, read as the exact
 * minimiser (grad E(x_{t+1}) = 0, implicit function theorem).  Given ax1 = dL/dx_{t+1} and av1 = dL/dv_{t+1}:
 *   H(x_{t+1}) lambda = ax1 + av1/h              (kinematic rows dropped), by Jacobi-preconditioned linear CG
 *   ax0 = dL/dx_t = M lambda - av1/h,   av0 = dL/dv_t = h M lambda   (x~ = x_t + h v_t + h^2 g; kinematic:
 *                                                                     ax0 = -av1/h, av0 = 0)
 *   dE[e] += -lambda_e . g_e / E_e               (the tet's elastic gradient g_e is linear in its Young's modulus)
 * CG runs to ||r|| <= tol ||b|| or max_iters iterations (sums in index order); *iters and *residual report them.
 */
int or_adjoint_step(const or_model *m, const double *x1, const double *ax1, const double *av1, double *ax0,
                    double *av0, double *dE, double tol, int32_t max_iters, int32_t *iters, double *residual)
{
    int32_t nv = m->p.nv;
    size_t n = 3 * (size_t)nv;
    double h = m->p.h;
    double *b = calloc(n, sizeof(double)), *lam = calloc(n, sizeof(double)), *r = calloc(n, sizeof(double));
    double *z = calloc(n, sizeof(double)), *p = calloc(n, sizeof(double)), *q = calloc(n, sizeof(double));
    double *g = calloc(n, sizeof(double)), *dg = calloc(n, sizeof(double));
    int st = OR_OK;
    if (!b || !lam || !r || !z || !p || !q || !g || !dg) { st = OR_ERR_OOM; goto done; }
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            size_t k = 3 * (size_t)i + a;
            b[k] = m->fixed[i] ? 0.0 : ax1[k] + av1[k] / h;
        }
    /* Jacobi preconditioner of the Hessian at x1 (the same rule as the iteration's, Sec. 4.2) */
    st = or_grad_diag(m, x1, x1, g, dg, NULL);
    if (st) goto done;
    double bb = 0.0;
    for (size_t k = 0; k < n; ++k) {
        int32_t i = (int32_t)(k / 3);
        dg[k] = m->fixed[i] ? 0.0 : (dg[k] > OR_JACOBI_FLOOR * m->mass[i] ? 1.0 / dg[k] : 1.0 / m->mass[i]);
        r[k] = b[k];
        z[k] = dg[k] * r[k];
        p[k] = z[k];
        bb += b[k] * b[k];
    }
    double rz = 0.0, rr = bb;
    for (size_t k = 0; k < n; ++k) rz += r[k] * z[k];
    int32_t it = 0;
    double bn = sqrt(bb);
    while (it < max_iters && sqrt(rr) > tol * bn && bn > 0.0) {
        st = or_hvp(m, x1, p, q);
        if (st) goto done;
        double pq = 0.0;
        for (size_t k = 0; k < n; ++k) pq += p[k] * q[k];
        if (!(pq != 0.0) || !isfinite(pq)) { st = OR_ERR_NONFINITE; set_err("CG breakdown"); goto done; }
        double al = rz / pq;
        double rz1 = 0.0;
        rr = 0.0;
        for (size_t k = 0; k < n; ++k) {
            lam[k] += al * p[k];
            r[k] -= al * q[k];
            z[k] = dg[k] * r[k];
            rz1 += r[k] * z[k];
            rr += r[k] * r[k];
        }
        double be = rz1 / rz;
        rz = rz1;
        for (size_t k = 0; k < n; ++k) p[k] = z[k] + be * p[k];
        ++it;
    }
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            size_t k = 3 * (size_t)i + a;
            double ml = m->fixed[i] ? 0.0 : m->mass[i] * lam[k];
            ax0[k] = ml - av1[k] / h;
            av0[k] = h * ml;
        }
    if (dE)
        for (int32_t e = 0; e < m->p.nt; ++e) {
            tet_terms T;
            st = tet_eval(m, e, x1, &T);
            if (st) { set_err("inverted tet"); goto done; }
            const int32_t *vi = m->tet + 4 * (size_t)e;
            double dPsi[9];
            for (int rr9 = 0; rr9 < 9; ++rr9) dPsi[rr9] = T.Psi1 * T.g1[rr9] + T.Psi2 * T.g2[rr9] + T.Psi3 * T.g3[rr9];
            double Ee = 2.0 * (1.0 + m->p.poisson) * m->mu[e];
            double s = 0.0;
            for (int qq = 0; qq < 12; ++qq) {
                double acc = 0.0;
                for (int rr9 = 0; rr9 < 9; ++rr9) acc += T.J[rr9][qq] * dPsi[rr9];
                s += lam[3 * (size_t)vi[qq / 3] + qq % 3] * T.scale * acc;
            }
            dE[e] -= s / Ee;
        }
    if (iters) *iters = it;
    if (residual) *residual = bn > 0.0 ? sqrt(rr) / bn : 0.0;
done:
    free(b); free(lam); free(r); free(z); free(p); free(q); free(g); free(dg);
    return st;
}
