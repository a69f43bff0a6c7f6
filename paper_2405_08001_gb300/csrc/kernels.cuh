// PNCG iteration kernels (Algorithm 1), templated on the element / barrier arithmetic type R:
//   R = double: the plain FP64 form;  R = float: FP32 element and barrier arithmetic on double vertex differences,
//   every reduction accumulated in double, the contact distance re-evaluated in double when d < 1e-3 dhat.
// Vertex state (x, xt, x~, v) is always double4_32a (w: unused / mass).  g, diag and p are R4 vectors.  The FP32 form
// also keeps float-float copies of the current and rest positions, so that its element kernels form vertex
// differences to ~2^-46 relative accuracy without FP64 arithmetic (FP64 throughput is low on this GPU).
#pragma once

#include "common.cuh"
#include "ffloat.cuh"
#include "geometry.cuh"
#include "material.cuh"

namespace pncg {

constexpr int VB = 128;   // threads per block, vertex kernels (148 blocks for the 18.8K-vertex bar: every SM busy)
constexpr int EB = 256;   // threads per block, element / pair kernels
static_assert(EB == SCATTER_CHUNK, "a tet block is one scatter chunk");

template <typename R> struct Dev {
    typedef typename V4<R>::T R4;
    int nv, nt, nfix;
    double4_32a *x, *xt, *xtil, *v, *xb;   // xtil.w = mass (free vertex) or -1 (kinematic)
    float4 *xh, *xl;                   // FP32 form: float-float copy of x (hi, lo); null in the FP64 form
    float4 *xbh;                       // FP32 form: xh at the last candidate build (displacement check)
    float4 *xth, *xtl;                 // FP32 form: float-float copy of xtil (hi with w = xtil.w, lo)
    const float *G0;                   // FP32 form: [14][nt] rest metric Dm^T Dm of each tet as float-float (six
                                       // heads, six tails), then det Dm as float-float
                                       // (hi of entries 00 01 02 11 12 22, then lo)
    float4 *tS;                        // FP32 form: [4][nt] of the last gradient pass per tet: S = 2 dPsi/dC and
                                       // C^-1 (entries 00 01 02 11 12 22 each), k1, k2, 0, 0 (tet_pHp_vec)
    R4 *g[2], *dg[2];                  // ping-pong by iteration parity; g.w = plane curvature kappa b'', dg.w = xtil.w
    R4 *p;
    R4 *pg, *pnext;                    // persistent form: P g of the current iteration, the next direction
    const double *mass;
    const int *fix_slot;               // [nv] target slot or -1
    const double *tgt;                 // staging [nfix][3] targets of the current step
    int has_tgt;
    // tets
    const int4 *tet;
    const R *Dm;                       // [9][nt] row-major D_m^-1 entries
    const R *hv;                       // [nt] h^2 V_e
    const R *escale;                   // [nt] E_e / E or nullptr
    R mu, lam;
    int model;                         // energy density: MAT_NH, MAT_SNH, MAT_FCR, MAT_ARAP (material.cuh)
    // contacts
    const int4 *cand;                  // candidates: PT (v, t0, t1, t2), EE (-1 - a0, a1, b0, b1)
    int cand_cap;
    Active<R> *act;
    // constants
    double h, dhat, kappa, eps, pad_r;
    double grav[3];
    int has_plane;
    double pn[3], po;
    int beta_rule, pnorm, iters;
    // segmented scatter: per (tet, corner) contributions [6][4 nt] and the vertex CSR
    R *contrib;
    const int *v2c_off, *v2c;          // v2c: 4*tet + corner
    int segmented;
    // block scatter: distinct vertices of each chunk of SCATTER_CHUNK tets and the chunk-local corner indices
    const int *cv_off, *cv;
    const ushort4 *tloc;
    int scatter_block;
    // colouring: tets sorted by colour (no two tets of a colour share a vertex); one kernel per colour
    const int *color_tets;
    int colored;
    // batching: nseg independent scenes (1 = none), the scene of each vertex, per-scene state and the per-scene
    // reduction accumulators ([3][nseg][8] sums, [3][nseg] maxima as bits; used round robin)
    int nseg;
    const int *vscene;
    int *cmark;                        // parts (split_objects = 2): 1 for the vertices of the step's collision parts
    SegCtl *seg;
    double *sacc;
    unsigned long long *smax;
    Ctrl *ctrl;
    double *part;                      // reduction partials
    double *trace;                     // [iters][TRACE_COLS]
};

template <typename R> __device__ inline void atomic_add4(typename V4<R>::T *p, R a, R b, R c);
template <> __device__ inline void atomic_add4<float>(float4 *p, float a, float b, float c)
{
    atomicAdd(p, make_float4(a, b, c, 0.0f));
}
template <> __device__ inline void atomic_add4<double>(double4_32a *p, double a, double b, double c)
{
    atomicAdd(&p->x, a);
    atomicAdd(&p->y, b);
    atomicAdd(&p->z, c);
}

__device__ inline void flag_error(Ctrl *c, uint32_t bits) { atomicOr(&c->err, bits); }

// Writes the FP32 form's float-float copy of x~ (vertex i; its w carries the mass slot of xtil.w).
template <typename R> __device__ inline void put_xt(const Dev<R> &D, int i, const double4_32a &XT)
{
    if constexpr (sizeof(R) == 4) {
        const ffl a = ff_split(XT.x), b = ff_split(XT.y), c = ff_split(XT.z);
        D.xth[i] = make_float4(a.h, b.h, c.h, (float)XT.w);
        D.xtl[i] = make_float4(a.l, b.l, c.l, 0.0f);
    }
}

// Writes vertex i's position (and, in the FP32 form, its float-float copy, whose head it returns).
template <typename R> __device__ inline float4 put_x(const Dev<R> &D, int i, const double4_32a &X)
{
    D.x[i] = X;
    if constexpr (sizeof(R) == 4) {
        const ffl a = ff_split(X.x), b = ff_split(X.y), c = ff_split(X.z);
        const float4 h = make_float4(a.h, b.h, c.h, 0.0f);
        D.xh[i] = h;
        D.xl[i] = make_float4(a.l, b.l, c.l, 0.0f);
        return h;
    } else {
        return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

// ------------------------------------------------------------------------------------------ vertex initialisation

// g = M (x - x~) and diag = m (Eq. E inertia term) plus the vertex / half-space barrier, written (not added) to
// the accumulators of parity `par`.  Kinematic vertices (xtil.w < 0) get zero inertia.
template <typename R>
__device__ inline void init_vertex(const Dev<R> &D, int i, const double4_32a &X, const double4_32a &XT, int par)
{
    const double m = XT.w;
    if constexpr (sizeof(R) == 4) {
        // the differences and the half-space distance and barrier in double, the rest in float (the values are
        // stored as floats): this runs for every vertex every iteration, and the FP64 pipes are scarce
        const float mm = m > 0.0 ? (float)m : 0.0f;
        float gx = mm * (float)(X.x - XT.x), gy = mm * (float)(X.y - XT.y), gz = mm * (float)(X.z - XT.z);
        float dx = mm, dy = mm, dz = mm, curv = 0.0f;
        if (D.has_plane) {
            const double d = D.pn[0] * X.x + D.pn[1] * X.y + D.pn[2] * X.z - D.po;
            if (d < D.dhat) {
                if (!(d > 0.0)) {
                    flag_error(D.ctrl, ERR_PENETRATION);
                } else {
                    // the barrier in float from the double d and d - dhat (a double log on every vertex in
                    // contact held its block back by 10-25 us per phase on this GPU's FP64 pipes), in double
                    // below 1e-3 dhat as for the pairs
                    float k1, k2;
                    if (d < 1e-3 * D.dhat) {
                        double b1, b2;
                        barrier_d12<double>(d, D.dhat, b1, b2);
                        k1 = (float)(D.kappa * b1); k2 = (float)(D.kappa * b2);
                    } else {
                        float b1, b2;
                        barrier_d12r<float>((float)d, (float)(d - D.dhat), (float)D.dhat, b1, b2);
                        k1 = (float)D.kappa * b1; k2 = (float)D.kappa * b2;
                    }
                    const float n0 = (float)D.pn[0], n1 = (float)D.pn[1], n2 = (float)D.pn[2];
                    gx += k1 * n0; gy += k1 * n1; gz += k1 * n2;
                    dx += k2 * n0 * n0; dy += k2 * n1 * n1; dz += k2 * n2 * n2;
                    curv = k2;
                }
            }
        }
        D.g[par][i] = mk4<R>(gx, gy, gz, curv);
        D.dg[par][i] = mk4<R>(dx, dy, dz, (float)m);
        return;
    }
    const double mm = m > 0.0 ? m : 0.0;
    double gx = mm * (X.x - XT.x), gy = mm * (X.y - XT.y), gz = mm * (X.z - XT.z);
    double dx = mm, dy = mm, dz = mm, curv = 0.0;
    if (D.has_plane) {
        double d = D.pn[0] * X.x + D.pn[1] * X.y + D.pn[2] * X.z - D.po;
        if (d < D.dhat) {
            if (!(d > 0.0)) {
                flag_error(D.ctrl, ERR_PENETRATION);
            } else {
                double b1, b2;
                barrier_d12<double>(d, D.dhat, b1, b2);
                double k1 = D.kappa * b1, k2 = D.kappa * b2;
                gx += k1 * D.pn[0]; gy += k1 * D.pn[1]; gz += k1 * D.pn[2];
                dx += k2 * D.pn[0] * D.pn[0]; dy += k2 * D.pn[1] * D.pn[1]; dz += k2 * D.pn[2] * D.pn[2];
                curv = k2;
            }
        }
    }
    D.g[par][i] = mk4<R>(R(gx), R(gy), R(gz), R(curv));
    D.dg[par][i] = mk4<R>(R(dx), R(dy), R(dz), R(m));
}

// init_vertex of the FP32 form after a position update, from the float-float copies of x (H + L, just written)
// and of x~: no FP64 arithmetic, except for a vertex whose float distance to the plane lies within dhat (plus that
// estimate's error bound), whose plane barrier is evaluated from the double position X as in init_vertex.
__device__ inline void init_vertex_ff(const Dev<float> &D, int i, const float4 &H, const float4 &L,
                                      const double4_32a &X, int par)
{
    const float4 TH = ldcg4(D.xth + i), TL = ldcg4(D.xtl + i);
    const float m = TH.w, mm = m > 0.0f ? m : 0.0f;
    float gx = mm * ff_val(ff_sub(H.x, L.x, TH.x, TL.x)), gy = mm * ff_val(ff_sub(H.y, L.y, TH.y, TL.y)),
          gz = mm * ff_val(ff_sub(H.z, L.z, TH.z, TL.z));
    float dx = mm, dy = mm, dz = mm, curv = 0.0f;
    if (D.has_plane) {
        // n . x - o in float from the heads: the dropped tails, the rounded n and o and the three roundings of the
        // FMAs are each at most 2^-24 of a value no larger than |x|_1 + |o| (n normalised), about 4e-7 of it in
        // all; the bound below leaves more than a factor of two
        const float n0 = (float)D.pn[0], n1 = (float)D.pn[1], n2 = (float)D.pn[2], o = (float)D.po;
        const float df = __fmaf_rn(n0, H.x, __fmaf_rn(n1, H.y, __fmaf_rn(n2, H.z, -o)));
        const float bound = 1e-6f * (fabsf(H.x) + fabsf(H.y) + fabsf(H.z) + fabsf(o));
        if (df < (float)D.dhat + bound) {
            const double d = D.pn[0] * X.x + D.pn[1] * X.y + D.pn[2] * X.z - D.po;
            if (d < D.dhat) {
                if (!(d > 0.0)) {
                    flag_error(D.ctrl, ERR_PENETRATION);
                } else {
                    float k1, k2;
                    if (d < 1e-3 * D.dhat) {
                        double b1, b2;
                        barrier_d12<double>(d, D.dhat, b1, b2);
                        k1 = (float)(D.kappa * b1); k2 = (float)(D.kappa * b2);
                    } else {
                        float b1, b2;
                        barrier_d12r<float>((float)d, (float)(d - D.dhat), (float)D.dhat, b1, b2);
                        k1 = (float)D.kappa * b1; k2 = (float)D.kappa * b2;
                    }
                    gx += k1 * n0; gy += k1 * n1; gz += k1 * n2;
                    dx += k2 * n0 * n0; dy += k2 * n1 * n1; dz += k2 * n2 * n2;
                    curv = k2;
                }
            }
        }
    }
    D.g[par][i] = make_float4(gx, gy, gz, curv);
    D.dg[par][i] = make_float4(dx, dy, dz, m);
}

// x += a p for vertex i (X in and out; a split as ah + al for the FP32 form) and the initialisation of the
// accumulators of parity par at the new x.  The FP32 form advances its float-float copy by float-float arithmetic (ff_axpy) beside
// the double state, so that the double update itself is its only FP64 work (FP64 issue is scarce on this GPU), and
// returns the new float head (the displacement check reads it).
template <typename R>
__device__ inline float4 update_vertex(const Dev<R> &D, int i, double4_32a &X, const typename V4<R>::T &P, double a,
                                       float ah, float al, const double4_32a &XT, int par)
{
    X.x += a * double(P.x); X.y += a * double(P.y); X.z += a * double(P.z);
    if constexpr (sizeof(R) == 4) {
        D.x[i] = X;
        float4 H = ldcg4(D.xh + i), L = ldcg4(D.xl + i);
        ff_axpy(H.x, L.x, ah, al, P.x);
        ff_axpy(H.y, L.y, ah, al, P.y);
        ff_axpy(H.z, L.z, ah, al, P.z);
        D.xh[i] = H;
        D.xl[i] = L;
        init_vertex_ff(D, i, H, L, X, par);
        return H;
    } else {
        put_x<R>(D, i, X);
        init_vertex<R>(D, i, X, XT, par);
        return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

__device__ inline double dist2(const double4_32a &a, const double4_32a &b)
{
    double x = a.x - b.x, y = a.y - b.y, z = a.z - b.z;
    return x * x + y * y + z * z;
}

// Squared displacement of vertex i since the last candidate build (float copies in the FP32 form).
template <typename R> __device__ inline double disp2(const Dev<R> &D, int i, const double4_32a &X)
{
    if constexpr (sizeof(R) == 4) {
        const float4 a = D.xh[i], b = D.xbh[i];
        const float x = a.x - b.x, y = a.y - b.y, z = a.z - b.z;
        return (double)(x * x + y * y + z * z);
    } else {
        return dist2(X, D.xb[i]);
    }
}

// Displacement bookkeeping shared by k_predict and k_update: when some vertex has moved pad_r / 2 since the last
// candidate build, request a rebuild (contacts can then not be missed: d changes by at most twice the largest
// vertex displacement).
template <typename R> __device__ inline void request_rebuild_if(const Dev<R> &D, double maxd2)
{
    double lim = 0.5 * D.pad_r * (1.0 - 1e-4);   // margin for the float displacement of the FP32 form
    if (maxd2 >= lim * lim && !D.ctrl->rebuild) {
        D.ctrl->cell_bits = 0u;
        D.ctrl->rebuild = 1;
    }
}

// a0: x^t = x; x~ = x + h v + h^2 gravity; kinematic vertices jump to their targets; init of iteration 0.
template <typename R>
__global__ void __launch_bounds__(VB) k_predict(Dev<R> D)
{
    __shared__ double sh[32 * 1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool skip = D.ctrl->err != 0u;
    double md2 = 0.0;
    if (i < D.nv && !skip) {
        double4_32a X = D.x[i], V = D.v[i];
        D.xt[i] = X;
        const int slot = D.fix_slot[i];
        double4_32a XT;
        if (slot >= 0) {
            if (D.has_tgt) {
                X.x = D.tgt[3 * slot]; X.y = D.tgt[3 * slot + 1]; X.z = D.tgt[3 * slot + 2];
            }
            XT = make_double4_32a(X.x, X.y, X.z, -1.0);
            put_x<R>(D, i, X);
        } else {
            const double h = D.h, h2 = D.h * D.h;
            XT = make_double4_32a(X.x + h * V.x + h2 * D.grav[0], X.y + h * V.y + h2 * D.grav[1],
                              X.z + h * V.z + h2 * D.grav[2], D.mass[i]);
        }
        D.xtil[i] = XT;
        put_xt<R>(D, i, XT);
        init_vertex<R>(D, i, X, XT, 0);
        md2 = disp2<R>(D, i, X);
    }
    double mx = block_max(md2, sh);
    double v1[1] = {mx};
    if (publish_partials<1>(v1, D.part, &D.ctrl->ticket[TK_PREDICT])) {
        double m = finish_max(D.part, 0, sh);
        if (threadIdx.x == 0) {
            Ctrl *c = D.ctrl;
            c->k = 0; c->n_rebuilds = 0; c->n_capped = 0; c->n_near64 = 0; c->iters_done = 0; c->converged = 0;
            c->n_active = 0; c->dE0 = 0.0; c->gPg_prev = 0.0;
            if (!skip) request_rebuild_if(D, m);
        }
    }
}

// ------------------------------------------------------------------------------------------ a2-a3: gradient + diag

// Per-tet Neo-Hookean quantities (Sec. 3.1): F = Ds Dm^-1, cofactor columns (gradient g3 of I3), I3 = det F.
template <typename R> struct TetF {
    R F[3][3];
    R cf[3][3];   // cf[a][b] = d det / d F_ab (columns f1 x f2, f2 x f0, f0 x f1)
    R J;
    R w[3][3];    // rows of Dm^-1 (vertex weights of x1, x2, x3; x0 gets minus their sum)
};

__device__ inline float comp(const float4 &v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// Edge vectors Ds[a][c] = x_{c+1,a} - x_{0,a}: from the double positions in the FP64 form, from the float-float
// positions (rounded once to float) in the FP32 form.
template <typename R> __device__ inline void tet_ds(const Dev<R> &D, const int4 &tv, R ds[3][3])
{
    if constexpr (sizeof(R) == 8) {
        const double4_32a X0 = ldcg4(D.x + tv.x), X1 = ldcg4(D.x + tv.y), X2 = ldcg4(D.x + tv.z), X3 = ldcg4(D.x + tv.w);
        ds[0][0] = X1.x - X0.x; ds[1][0] = X1.y - X0.y; ds[2][0] = X1.z - X0.z;
        ds[0][1] = X2.x - X0.x; ds[1][1] = X2.y - X0.y; ds[2][1] = X2.z - X0.z;
        ds[0][2] = X3.x - X0.x; ds[1][2] = X3.y - X0.y; ds[2][2] = X3.z - X0.z;
    } else {
        const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
        const float4 h0 = ldcg4(D.xh + vid[0]), l0 = ldcg4(D.xl + vid[0]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 h = ldcg4(D.xh + vid[c + 1]), l = ldcg4(D.xl + vid[c + 1]);
#pragma unroll
            for (int a = 0; a < 3; ++a) ds[a][c] = ff_val(ff_sub(comp(h, a), comp(l, a), comp(h0, a), comp(l0, a)));
        }
    }
}

template <typename R> __device__ inline void load_w(const Dev<R> &D, int e, R w[3][3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) w[r][c] = D.Dm[(3 * r + c) * D.nt + e];
}

template <typename R> __device__ inline void tet_F_from(const R ds[3][3], TetF<R> &T)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) T.F[a][b] = ds[a][0] * T.w[0][b] + ds[a][1] * T.w[1][b] + ds[a][2] * T.w[2][b];
    T.cf[0][0] = T.F[1][1] * T.F[2][2] - T.F[2][1] * T.F[1][2];
    T.cf[1][0] = T.F[2][1] * T.F[0][2] - T.F[0][1] * T.F[2][2];
    T.cf[2][0] = T.F[0][1] * T.F[1][2] - T.F[1][1] * T.F[0][2];
    T.cf[0][1] = T.F[1][2] * T.F[2][0] - T.F[2][2] * T.F[1][0];
    T.cf[1][1] = T.F[2][2] * T.F[0][0] - T.F[0][2] * T.F[2][0];
    T.cf[2][1] = T.F[0][2] * T.F[1][0] - T.F[1][2] * T.F[0][0];
    T.cf[0][2] = T.F[1][0] * T.F[2][1] - T.F[2][0] * T.F[1][1];
    T.cf[1][2] = T.F[2][0] * T.F[0][1] - T.F[0][0] * T.F[2][1];
    T.cf[2][2] = T.F[0][0] * T.F[1][1] - T.F[1][0] * T.F[0][1];
    T.J = T.F[0][0] * T.cf[0][0] + T.F[1][0] * T.cf[1][0] + T.F[2][0] * T.cf[2][0];
}

template <typename R> __device__ inline void tet_F(const Dev<R> &D, int e, const int4 &tv, TetF<R> &T)
{
    R ds[3][3];
    tet_ds<R>(D, tv, ds);
    load_w<R>(D, e, T.w);
    tet_F_from<R>(ds, T);
}

template <typename R> __device__ inline void tet_material(const Dev<R> &D, int e, R &mu, R &lam)
{
    mu = D.mu;
    lam = D.lam;
    if (D.escale) { R s = D.escale[e]; mu *= s; lam *= s; }
}

// The per-tet constants a gradient evaluation streams in (coalesced, structure-of-arrays in memory): indices,
// D_m^-1, h^2 V, the Young's modulus scale and, in the FP32 form, the float-float rest metric.
template <typename R> struct TetIn {
    int4 tv;
    R w[3][3];
    R hv, es;
    float g0[14];   // FP32 form: rest metric entries 00 01 02 11 12 22, heads then tails; det Dm head, tail
};
template <typename R> __device__ inline void load_tet_in(const Dev<R> &D, int e, TetIn<R> &in)
{
    in.tv = D.tet[e];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) in.w[r][c] = D.Dm[(3 * r + c) * D.nt + e];
    in.hv = D.hv[e];
    in.es = D.escale ? D.escale[e] : R(1);
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int q = 0; q < 14; ++q) in.g0[q] = D.G0[q * D.nt + e];
    }
}

// Small symmetric 3x3 helpers of the FP32 corotated path.
__device__ inline void sym_inv3f(const float X[3][3], float Xi[3][3])
{
    const float c00 = X[1][1] * X[2][2] - X[1][2] * X[1][2], c01 = X[0][2] * X[1][2] - X[0][1] * X[2][2];
    const float c02 = X[0][1] * X[1][2] - X[0][2] * X[1][1], c11 = X[0][0] * X[2][2] - X[0][2] * X[0][2];
    const float c12 = X[0][1] * X[0][2] - X[0][0] * X[1][2], c22 = X[0][0] * X[1][1] - X[0][1] * X[0][1];
    const float id = 1.0f / (X[0][0] * c00 + X[0][1] * c01 + X[0][2] * c02);
    Xi[0][0] = c00 * id; Xi[1][1] = c11 * id; Xi[2][2] = c22 * id;
    Xi[0][1] = Xi[1][0] = c01 * id;
    Xi[0][2] = Xi[2][0] = c02 * id;
    Xi[1][2] = Xi[2][1] = c12 * id;
}
__device__ inline float quad3f(const float M[3][3], float a0, float a1, float a2)
{
    return a0 * (M[0][0] * a0 + M[0][1] * a1 + M[0][2] * a2) + a1 * (M[1][0] * a0 + M[1][1] * a1 + M[1][2] * a2) +
           a2 * (M[2][0] * a0 + M[2][1] * a1 + M[2][2] * a2);
}

// The corotated densities' FP32 terms of one tet, computed out of line (arguments and result by value) so that
// their temporaries stay out of the register budget of the passes that run the Neo-Hookean path.
struct CorotIn {
    float A[3][3], F[3][3], cf[3][3], w[3][3];   // C - I, F, cof(F), rows of Dm^-1
    float J, Jm1, mu, lam, hv;
    int fcr;                                      // 1: FCR (the lambda (J - 1)^2 / 2 term), 0: ARAP
};
struct CorotOut {
    float P[3][3];    // first Piola-Kirchhoff stress times h^2 V
    float dv[4][3];   // h^2 V Psi_1 d2I1 on the diagonal, per vertex and component
    float rec[16];    // p^T H p record: R (9, row-major), Dq (6: 00 01 02 11 12 22), J - 1
    float Psi33;
};

// U - I = V = sqrt(I + A) - I of the stretch from the metric change A = C - I (symmetric), by Newton's iteration
// for the principal square root, X <- (X + X^-1 (I + A)) / 2, written for V from V = A / 2 (which bounds the root
// from above, so the iteration decreases monotonically): V <- V + (I + V)^-1 (A - 2 V - V^2) / 2, symmetrised.  The
// residual A - 2 V - V^2 is formed from the accurate A, so V keeps its relative accuracy for small strains where the
// I2 / I1 parts of the stress cancel.  Quadratic convergence; at most 8 steps (5 for stretches up to 10).
__device__ inline void stretch_minus_identity(const float A[3][3], float V[3][3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) V[a][b] = 0.5f * A[a][b];
    for (int it = 0; it < 8; ++it) {
        float X[3][3], Xi[3][3], r[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                X[a][b] = V[a][b] + (a == b ? 1.0f : 0.0f);
                r[a][b] = A[a][b] - 2.0f * V[a][b] - (V[a][0] * V[0][b] + V[a][1] * V[1][b] + V[a][2] * V[2][b]);
            }
        sym_inv3f(X, Xi);
        float dmax = 0.0f, vmax = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
                const float d = 0.25f * (Xi[a][0] * r[0][b] + Xi[a][1] * r[1][b] + Xi[a][2] * r[2][b] +
                                         r[a][0] * Xi[0][b] + r[a][1] * Xi[1][b] + r[a][2] * Xi[2][b]);
                V[a][b] += d;
                V[b][a] = V[a][b];
                dmax = fmaxf(dmax, fabsf(d));
                vmax = fmaxf(vmax, fabsf(V[a][b]));
            }
        if (dmax <= 1e-7f * vmax) break;
    }
}

// FCR, ARAP in the FP32 form (Psi_1 = -2 mu, 2 Psi_2 = 2 mu; FCR: Psi_3 = lambda (J - 1), Psi_33 = lambda).  With the
// stretch U (F = R U) and V = U - I, F^T P = 2 mu U (U - I) + Psi_3 J I = 2 mu (V + V^2) + lambda J (J - 1) I, so
// P = F^-T M as for the other densities.  R = F (I + V)^-1; the twist modes of d2I1(F)[dF, dF] = a^T (tr(U) I -
// U)^-1 a (a = axial(R^T dF - dF^T R); derivation in material.cuh) with tr(U) I - U = N = (2 + tr V) I - V; the
// diagonal takes a = w x rho (rho = R^T e_c), p^T H p the difference Dq = I/2 - N^-1 = N^-1 (tr V I - V) / 2, which
// is small near a rotation and formed here without cancellation.
static __device__ __noinline__ CorotOut corot_terms(CorotIn ci)
{
    CorotOut co;
    float V[3][3];
    stretch_minus_identity(ci.A, V);
    co.Psi33 = ci.fcr ? ci.lam : 0.0f;
    const float pj = ci.fcr ? ci.lam * ci.J * ci.Jm1 : 0.0f;
    float M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            M[a][b] = 2.0f * ci.mu * (V[a][b] + V[a][0] * V[0][b] + V[a][1] * V[1][b] + V[a][2] * V[2][b]) +
                      (a == b ? pj : 0.0f);
    const float sj = ci.hv / ci.J;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) co.P[a][b] = sj * (ci.cf[a][0] * M[0][b] + ci.cf[a][1] * M[1][b] + ci.cf[a][2] * M[2][b]);
    float X[3][3], Xi[3][3], N[3][3], Ni[3][3], W[3][3], Rm[3][3], Dq[3][3];
    const float tv = V[0][0] + V[1][1] + V[2][2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            X[a][b] = V[a][b] + (a == b ? 1.0f : 0.0f);
            N[a][b] = (a == b ? 2.0f + tv : 0.0f) - V[a][b];
            W[a][b] = (a == b ? tv : 0.0f) - V[a][b];
        }
    sym_inv3f(X, Xi);
    sym_inv3f(N, Ni);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Rm[a][b] = ci.F[a][0] * Xi[0][b] + ci.F[a][1] * Xi[1][b] + ci.F[a][2] * Xi[2][b];
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b)
            Dq[a][b] = Dq[b][a] = 0.25f * (Ni[a][0] * W[0][b] + Ni[a][1] * W[1][b] + Ni[a][2] * W[2][b] +
                                           W[a][0] * Ni[0][b] + W[a][1] * Ni[1][b] + W[a][2] * Ni[2][b]);
    const float ps1 = -2.0f * ci.mu * ci.hv;   // h^2 V Psi_1
    for (int i = 0; i < 4; ++i) {
        float w[3];
        for (int b = 0; b < 3; ++b) w[b] = i == 0 ? -(ci.w[0][b] + ci.w[1][b] + ci.w[2][b]) : ci.w[i - 1][b];
        for (int a = 0; a < 3; ++a) {
            const float r0 = Rm[a][0], r1 = Rm[a][1], r2 = Rm[a][2];
            co.dv[i][a] = ps1 * quad3f(Ni, w[1] * r2 - w[2] * r1, w[2] * r0 - w[0] * r2, w[0] * r1 - w[1] * r0);
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) co.rec[3 * a + b] = Rm[a][b];
    co.rec[9] = Dq[0][0]; co.rec[10] = Dq[0][1]; co.rec[11] = Dq[0][2];
    co.rec[12] = Dq[1][1]; co.rec[13] = Dq[1][2]; co.rec[14] = Dq[2][2];
    co.rec[15] = ci.Jm1;
    return co;
}

// p^T H p of one tet of a corotated density in the FP32 form, from the record of its gradient pass:
//   2 mu (|dF|^2 - a^T N^-1 a) = 2 mu (|sym K|^2 + a^T Dq a),  K = R^T dF,  a = axial(K - K^T)
// (|skew K|^2 = |a|^2 / 2): a direction that rotates the tet gives sym K = 0 and the small Dq, so the terms that
// cancel for it never meet in float; FCR adds lambda (cof(F) : dF)^2 + lambda (J - 1) d2det(F)[dF, dF].
struct CorotPIn {
    float rec[16];
    float dF[3][3], F[3][3], cf[3][3];
    float mu, lam;
    int fcr;
};
static __device__ __noinline__ float corot_pHp(CorotPIn ci)
{
    float K[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            K[a][b] = ci.rec[a] * ci.dF[0][b] + ci.rec[3 + a] * ci.dF[1][b] + ci.rec[6 + a] * ci.dF[2][b];
    float s2 = 0.0f;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) { const float sk = 0.5f * (K[a][b] + K[b][a]); s2 += sk * sk; }
    const float Dq[3][3] = {{ci.rec[9], ci.rec[10], ci.rec[11]}, {ci.rec[10], ci.rec[12], ci.rec[13]},
                            {ci.rec[11], ci.rec[13], ci.rec[14]}};
    float q = 2.0f * ci.mu * (s2 + quad3f(Dq, K[2][1] - K[1][2], K[0][2] - K[2][0], K[1][0] - K[0][1]));
    if (ci.fcr) {
        float g3 = 0.0f;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) g3 += ci.cf[a][b] * ci.dF[a][b];
        const v3<float> f0 = mkv(ci.F[0][0], ci.F[1][0], ci.F[2][0]), f1 = mkv(ci.F[0][1], ci.F[1][1], ci.F[2][1]),
                        f2 = mkv(ci.F[0][2], ci.F[1][2], ci.F[2][2]);
        const v3<float> d0 = mkv(ci.dF[0][0], ci.dF[1][0], ci.dF[2][0]), d1 = mkv(ci.dF[0][1], ci.dF[1][1], ci.dF[2][1]),
                        d2 = mkv(ci.dF[0][2], ci.dF[1][2], ci.dF[2][2]);
        const float h3 = 2.0f * (dot(d0, cross(d1, f2)) + dot(d0, cross(f1, d2)) + dot(f0, cross(d1, d2)));
        q += ci.lam * (g3 * g3 + ci.rec[15] * h3);
    }
    return q;
}

// First Piola-Kirchhoff stress of the FP32 form, evaluated from the metric change so that it stays accurate for
// small strains under any rotation.  With C = F^T F and a density of I2 and I3 (Sec. 3.1: NH or SNH) written in C,
//   P = F^-T (mu (C - I) + (mu + Psi_3 J) I),   C - I = Dm^-T (Ds^T Ds - Dm^T Dm) Dm^-1,
// which equals mu F + Psi_3 cof(F) (the I2/I3 form) exactly; mu + Psi_3 J is lambda log J for NH.  The metric
// change G = Ds^T Ds - Dm^T Dm is accumulated in float-float from the float-float current positions and the tet's
// float-float rest metric, and G W is formed with compensated products, so that rounding never acts on the parts
// that cancel.  J - 1 = (det Ds - det Dm) / det Dm comes from det Ds in float-float and the tet's
// float-float det Dm: under large shear a nearly incompressible tet keeps J near 1 while the entries of C - I are
// of order one, and det C - 1 expanded in those entries cancels (lambda log J then carried about 1e-5 of the
// stress).  F^-T = cof(F) / J.  Returns false (and flags the error) when det F <= 0.  Also returns Psi_33 for the
// diagonal.
template <bool CO>
__device__ inline bool tet_stress_metric(const Dev<float> &D, const TetIn<float> &in, TetF<float> &T, float P[3][3],
                                         float &Psi33, int e, CorotOut *cr = nullptr)
{
    const int4 tv = in.tv;
    const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
    float4 xh[4], xl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { xh[k] = ldcg4(D.xh + vid[k]); xl[k] = ldcg4(D.xl + vid[k]); }
    float g0h[6], g0l[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) { g0h[q] = in.g0[q]; g0l[q] = in.g0[6 + q]; }
    ffl ds[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) ds[a][c] = ff_sub(comp(xh[c + 1], a), comp(xl[c + 1], a), comp(xh[0], a), comp(xl[0], a));
    ffl G[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const int q = (i == 0 ? j : (i == 1 ? 2 + j : 5));   // 00 01 02 11 12 22
            ffacc acc = ffacc::prod(ds[0][i], ds[0][j]);
#pragma unroll
            for (int a = 1; a < 3; ++a) acc.add_prod(ds[a][i], ds[a][j], 1.0f);
            acc.sub_ff(g0h[q], g0l[q]);
            G[i][j] = G[j][i] = acc.ff();
        }
    float dsf[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) dsf[a][c] = ff_val(ds[a][c]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) T.w[r][c] = in.w[r][c];
    tet_F_from<float>(dsf, T);
    if (!(T.J > 0.0f)) { flag_error(D.ctrl, ERR_INVERTED); return false; }
    // A = C - I = W^T G W with W = Dm^-1 (T.w[r][c] = W_rc): G W with compensated (Dot2) products from the
    // float-float G, rounded once, then W^T (G W) in float.  The terms are up to cond(Dm)^2 times larger than A and
    // cancel; in plain float from a rounded G that cost about 1e-6 of the stress on strongly sheared tets
    // (compensating the second product as well gained nothing measurable)
    float GW[3][3], A[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            ffacc acc = ffacc::prod_f(G[i][0], T.w[0][b]);
#pragma unroll
            for (int j = 1; j < 3; ++j) acc.add_prod_f(G[i][j], T.w[j][b]);
            GW[i][b] = acc.value();
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) A[a][b] = A[b][a] = T.w[0][a] * GW[0][b] + T.w[1][a] * GW[1][b] + T.w[2][a] * GW[2][b];
    // J - 1 from det Ds (float-float; the edge vectors ds[a][c] = component a of edge c) and det Dm
    float Jm1;
    {
        ffn a[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) a[r][c] = ffn(ds[r][c].h, ds[r][c].l);
        const ffn det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                        a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                        a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
        const ffn dd = det - ffn(in.g0[12], in.g0[13]);
        Jm1 = __fdiv_rn(__fadd_rn(dd.h, dd.l), in.g0[12]);
    }
    const float J = 1.0f + Jm1;
    if (!(J > 0.0f)) { flag_error(D.ctrl, ERR_INVERTED); return false; }
    const float detC = J * J;
    const float mu = D.mu * in.es, lam = D.lam * in.es;
    if (CO && (D.model == MAT_FCR || D.model == MAT_ARAP)) {
        CorotIn ci;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) { ci.A[a][b] = A[a][b]; ci.F[a][b] = T.F[a][b]; ci.cf[a][b] = T.cf[a][b]; ci.w[a][b] = T.w[a][b]; }
        ci.J = J; ci.Jm1 = Jm1; ci.mu = mu; ci.lam = lam; ci.hv = in.hv; ci.fcr = D.model == MAT_FCR;
        const CorotOut co = corot_terms(ci);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) P[a][b] = co.P[a][b];
        Psi33 = co.Psi33;
        if (cr) *cr = co;
        if (e >= 0) {   // R, Dq and J - 1 for the p^T H p pass
            const size_t n = (size_t)D.nt;
            D.tS[e] = make_float4(co.rec[0], co.rec[1], co.rec[2], co.rec[3]);
            D.tS[n + e] = make_float4(co.rec[4], co.rec[5], co.rec[6], co.rec[7]);
            D.tS[2 * n + e] = make_float4(co.rec[8], co.rec[9], co.rec[10], co.rec[11]);
            D.tS[3 * n + e] = make_float4(co.rec[12], co.rec[13], co.rec[14], co.rec[15]);
        }
        return true;
    }
    // mJ = mu + Psi_3 J: lambda log J (NH), (J - 1)(lambda J - mu) (SNH)
    // k1 = J (Psi_33 J + Psi_3) / 4, k2 = -Psi_3 J / 2: the coefficients of p^T H p in C (tet_pHp_vec)
    float mJ, k1, k2;
    if (D.model == MAT_SNH) {
        mJ = Jm1 * (lam * J - mu);
        Psi33 = lam;
        k1 = 0.25f * J * (lam * (J + Jm1) - mu);
        k2 = 0.5f * J * (mu - lam * Jm1);
    } else {
        const float L = log1pf(Jm1);                                                // log J
        mJ = lam * L;
        Psi33 = (mu + lam * (1.0f - L)) / detC;
        k1 = 0.25f * lam;
        k2 = 0.5f * (mu - lam * L);
    }
    // C^-1 = cof(C) / det C (C symmetric)
    const float c00 = 1.0f + A[0][0], c11 = 1.0f + A[1][1], c22 = 1.0f + A[2][2];
    const float ic = 1.0f / detC;
    float Ci[3][3];
    Ci[0][0] = (c11 * c22 - A[1][2] * A[1][2]) * ic;
    Ci[1][1] = (c00 * c22 - A[0][2] * A[0][2]) * ic;
    Ci[2][2] = (c00 * c11 - A[0][1] * A[0][1]) * ic;
    Ci[0][1] = Ci[1][0] = (A[0][2] * A[1][2] - A[0][1] * c22) * ic;
    Ci[0][2] = Ci[2][0] = (A[0][1] * A[1][2] - A[0][2] * c11) * ic;
    Ci[1][2] = Ci[2][1] = (A[0][1] * A[0][2] - A[1][2] * c00) * ic;
    float M[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[a][b] = mu * A[a][b] + (a == b ? mJ : 0.0f);
    float S[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) S[a][b] = Ci[a][0] * M[0][b] + Ci[a][1] * M[1][b] + Ci[a][2] * M[2][b];
    // P = F^-T M with F^-T = cof(F) / J (T.cf[a][c] is the cofactor of F_ac)
    const float sc = in.hv, sj = sc / J;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P[a][b] = sj * (T.cf[a][0] * M[0][b] + T.cf[a][1] * M[1][b] + T.cf[a][2] * M[2][b]);
    if (e >= 0) {   // S (symmetric: C^-1 commutes with C - I), C^-1, k1, k2 for the p^T H p pass
        const size_t n = (size_t)D.nt;
        D.tS[e] = make_float4(S[0][0], 0.5f * (S[0][1] + S[1][0]), 0.5f * (S[0][2] + S[2][0]), S[1][1]);
        D.tS[n + e] = make_float4(0.5f * (S[1][2] + S[2][1]), S[2][2], Ci[0][0], Ci[0][1]);
        D.tS[2 * n + e] = make_float4(Ci[0][2], Ci[1][1], Ci[1][2], Ci[2][2]);
        D.tS[3 * n + e] = make_float4(k1, k2, 0.0f, 0.0f);
    }
    return true;
}

// Element gradient and Jacobi diagonal (Sec. 3.1 split; no density here has Psi_11 or Psi_22 terms and the H3
// term has a zero diagonal, so diag_i[a] = h^2 V (2 Psi_2 |w_i|^2 + Psi_33 (cof(F) w_i)_a^2 + Psi_1 d2I1 entry)).  The contributions go to the
// per-(tet, corner) buffer (segmented scatter), to the block's shared accumulators sacc ([6][SCATTER_MAXU],
// indexed by the chunk-local vertex; block scatter) or straight to the global accumulators.
template <typename R, bool CO = false>
__device__ inline bool tet_grad_eval(const Dev<R> &D, const TetIn<R> &in, R gv[4][3], R dv[4][3], int e = -1)
{
    const int4 tv = in.tv;
    TetF<R> T;
    R P[3][3], Psi33;
    const R sc = in.hv;
    const R mu = D.mu * in.es, lam = D.lam * in.es;
    R c2 = mu;        // 2 Psi_2
    R Psi1 = R(0);    // the I1 term (FCR, ARAP)
    if constexpr (sizeof(R) == 4) {
        if constexpr (CO) {
            CorotOut cr;
            if (!tet_stress_metric<true>(D, in, T, P, Psi33, e, &cr)) return false;
            if (D.model == MAT_FCR || D.model == MAT_ARAP) {   // Psi_1 d2I1 on the diagonal
                c2 = R(2) * mu;
                Psi1 = R(-2) * mu;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int a = 0; a < 3; ++a) dv[i][a] = cr.dv[i][a];
            }
        } else {
            if (!tet_stress_metric<false>(D, in, T, P, Psi33, e)) return false;
        }
    } else {
        R ds[3][3];
        tet_ds<R>(D, tv, ds);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) T.w[r][c] = in.w[r][c];
        tet_F_from<R>(ds, T);
        if (!(T.J > R(0))) { flag_error(D.ctrl, ERR_INVERTED); return false; }
        const MatTerms<R> mt = mat_terms<R>(D.model, mu, lam, T.J);
        Psi33 = mt.Psi33;
        c2 = mt.c2;
        Psi1 = mt.Psi1;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) P[a][b] = sc * (c2 * T.F[a][b] + mt.Psi3 * T.cf[a][b]);
        if (Psi1 != R(0)) {   // FCR, ARAP: Psi_1 R in the stress, Psi_1 d2I1 on the diagonal
            Polar pol;
            polar_of(T.F, pol);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) P[a][b] += sc * Psi1 * pol.R[a][b];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                double w[3];
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    w[b] = i == 0 ? -(T.w[0][b] + T.w[1][b] + T.w[2][b]) : T.w[i - 1][b];
#pragma unroll
                for (int a = 0; a < 3; ++a) dv[i][a] = sc * Psi1 * polar_h1_diag(pol, w, a);
            }
        }
    }
    const bool i1 = Psi1 != R(0);
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        const R *w = T.w[i - 1];
        const R ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gv[i][a] = P[a][0] * w[0] + P[a][1] * w[1] + P[a][2] * w[2];
            const R cw = T.cf[a][0] * w[0] + T.cf[a][1] * w[1] + T.cf[a][2] * w[2];
            dv[i][a] = (i1 ? dv[i][a] : R(0)) + sc * (c2 * ww + Psi33 * cw * cw);
        }
    }
    {
        R w0[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) w0[b] = -(T.w[0][b] + T.w[1][b] + T.w[2][b]);
        const R ww = w0[0] * w0[0] + w0[1] * w0[1] + w0[2] * w0[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gv[0][a] = -(gv[1][a] + gv[2][a] + gv[3][a]);
            const R cw = T.cf[a][0] * w0[0] + T.cf[a][1] * w0[1] + T.cf[a][2] * w0[2];
            dv[0][a] = (i1 ? dv[0][a] : R(0)) + sc * (c2 * ww + Psi33 * cw * cw);
        }
    }
    return true;
}

template <typename R, bool CO = false>
__device__ inline void tet_grad(const Dev<R> &D, int e, int par, const TetIn<R> &in, R *sacc = nullptr)
{
    const int4 tv = in.tv;
    R gv[4][3], dv[4][3];
    if (!tet_grad_eval<R, CO>(D, in, gv, dv, e)) return;
    if (D.segmented) {
        const int q0 = 4 * e;
        const int n4 = 4 * D.nt;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                D.contrib[a * n4 + q0 + i] = gv[i][a];
                D.contrib[(3 + a) * n4 + q0 + i] = dv[i][a];
            }
        return;
    }
    if (sacc) {
        const ushort4 lc = D.tloc[e];
        const int loc[4] = {lc.x, lc.y, lc.z, lc.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                atomicAdd(sacc + a * SCATTER_MAXU + loc[i], gv[i][a]);
                atomicAdd(sacc + (3 + a) * SCATTER_MAXU + loc[i], dv[i][a]);
            }
        return;
    }
    const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
    if (D.colored) {   // no other tet of this launch's colour touches these vertices: plain read-modify-write
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            typename V4<R>::T G = D.g[par][vid[i]], Dg = D.dg[par][vid[i]];
            G.x += gv[i][0]; G.y += gv[i][1]; G.z += gv[i][2];
            Dg.x += dv[i][0]; Dg.y += dv[i][1]; Dg.z += dv[i][2];
            D.g[par][vid[i]] = G;
            D.dg[par][vid[i]] = Dg;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        atomic_add4<R>(&D.g[par][vid[i]], gv[i][0], gv[i][1], gv[i][2]);
        atomic_add4<R>(&D.dg[par][vid[i]], dv[i][0], dv[i][1], dv[i][2]);
    }
}

// Colouring scatter: the tets of one colour (positions t0 .. t0 + n of the colour order), one thread each.  Dc is
// D with the per-tet inputs (tet, Dm, hv, escale, G0) in colour order, so that the loads of a colour stay
// coalesced; the record of the p^T H p pass is written at the tet's own index color_tets[q].
template <typename R, bool CO = false>
__global__ void __launch_bounds__(EB) k_grad_color(Dev<R> D, Dev<R> Dc, int par, int t0, int n)
{
    const int q = t0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (q >= t0 + n) return;
    TetIn<R> in;
    load_tet_in<R>(Dc, q, in);
    tet_grad<R, CO>(D, D.color_tets[q], par, in);
}

// The colour-ordered copies of the per-tet inputs (once, at setup): position q holds tet color_tets[q].
template <typename R>
__global__ void k_color_gather(Dev<R> D, int4 *tet, R *Dm, R *hv, R *es, float *G0)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= D.nt) return;
    const size_t n = (size_t)D.nt;
    const int e = D.color_tets[q];
    tet[q] = D.tet[e];
    for (int k = 0; k < 9; ++k) Dm[k * n + q] = D.Dm[k * n + e];
    hv[q] = D.hv[e];
    if (es) es[q] = D.escale[e];
    if (G0)
        for (int k = 0; k < 14; ++k) G0[k * n + q] = D.G0[k * n + e];
}

// The tets of chunk ch (SCATTER_CHUNK consecutive tets, one per thread of the block): gradient and diagonal,
// block-scattered when the chunk's distinct vertices fit the shared accumulators.  Called by all threads of a
// block with a block-uniform ch.
template <typename R, bool CO = false>
__device__ inline void tet_grad_chunk(const Dev<R> &D, int ch, int par, R *sacc)
{
    const int e = ch * SCATTER_CHUNK + (int)threadIdx.x;
    int u0 = 0, nu = 0;
    if (D.scatter_block) { u0 = D.cv_off[ch]; nu = D.cv_off[ch + 1] - u0; }
    const bool blk = D.scatter_block && nu <= SCATTER_MAXU;
    if (blk) {
        for (int q = threadIdx.x; q < 6 * SCATTER_MAXU; q += blockDim.x) {
            if ((q % SCATTER_MAXU) < nu) sacc[q] = R(0);
        }
        __syncthreads();
    }
    if (e < D.nt) {
        TetIn<R> in;
        load_tet_in<R>(D, e, in);
        tet_grad<R, CO>(D, e, par, in, blk ? sacc : nullptr);
    }
    if (blk) {
        __syncthreads();
        for (int u = threadIdx.x; u < nu; u += blockDim.x) {
            const int v = D.cv[u0 + u];
            atomic_add4<R>(&D.g[par][v], sacc[u], sacc[SCATTER_MAXU + u], sacc[2 * SCATTER_MAXU + u]);
            atomic_add4<R>(&D.dg[par][v], sacc[3 * SCATTER_MAXU + u], sacc[4 * SCATTER_MAXU + u], sacc[5 * SCATTER_MAXU + u]);
        }
        __syncthreads();
    }
}

// Closest-point coefficients and t of a candidate.  Relative coordinates come from the double positions (FP64
// form, and the FP32 form's double re-evaluation) or from the float-float positions (FP32 form).
template <typename R>
__device__ inline R pair_geom(bool ee, const double4_32a &X0, const double4_32a &X1, const double4_32a &X2, const double4_32a &X3,
                              R c[4], v3<R> &t)
{
    if (!ee) {
        return pt_coeffs<R>(rel<R>(X0.x, X0.y, X0.z, X1.x, X1.y, X1.z), rel<R>(X2.x, X2.y, X2.z, X1.x, X1.y, X1.z),
                            rel<R>(X3.x, X3.y, X3.z, X1.x, X1.y, X1.z), c, t);
    }
    return ee_coeffs<R>(rel<R>(X0.x, X0.y, X0.z, X2.x, X2.y, X2.z), rel<R>(X1.x, X1.y, X1.z, X2.x, X2.y, X2.z),
                        rel<R>(X3.x, X3.y, X3.z, X2.x, X2.y, X2.z), c, t);
}

__device__ inline v3<float> rel_ff(const Dev<float> &D, int a, int b)
{
    const float4 ha = ldcg4(D.xh + a), la = ldcg4(D.xl + a), hb = ldcg4(D.xh + b), lb = ldcg4(D.xl + b);
    return mkv(ff_val(ff_sub(ha.x, la.x, hb.x, lb.x)), ff_val(ff_sub(ha.y, la.y, hb.y, lb.y)),
               ff_val(ff_sub(ha.z, la.z, hb.z, lb.z)));
}

__device__ inline float pair_geom_ff(const Dev<float> &D, bool ee, const int4 &v, float c[4], v3<float> &t)
{
    if (!ee) return pt_coeffs<float>(rel_ff(D, v.x, v.y), rel_ff(D, v.z, v.y), rel_ff(D, v.w, v.y), c, t);
    return ee_coeffs<float>(rel_ff(D, v.x, v.z), rel_ff(D, v.y, v.z), rel_ff(D, v.w, v.z), c, t);
}

// The same geometry in float-float arithmetic, for the pairs the float pass found active: the float distance
// loses about log2(|x_i - x_j| / d) bits, and the barrier terms (B = kappa b'/d < 0 against A > 0) often cancel in
// p^T H p and in the diagonal.
__device__ inline v3<ffn> rel_ffn(const Dev<float> &D, int a, int b)
{
    const float4 ha = ldcg4(D.xh + a), la = ldcg4(D.xl + a), hb = ldcg4(D.xh + b), lb = ldcg4(D.xl + b);
    const ffl x = ff_sub(ha.x, la.x, hb.x, lb.x), y = ff_sub(ha.y, la.y, hb.y, lb.y), z = ff_sub(ha.z, la.z, hb.z, lb.z);
    return mkv(ffn(x.h, x.l), ffn(y.h, y.l), ffn(z.h, z.l));
}
__device__ inline ffn pair_geom_ffn(const Dev<float> &D, bool ee, const int4 &v, ffn c[4], v3<ffn> &t)
{
    if (!ee) return pt_coeffs<ffn>(rel_ffn(D, v.x, v.y), rel_ffn(D, v.z, v.y), rel_ffn(D, v.w, v.y), c, t);
    return ee_coeffs<ffn>(rel_ffn(D, v.x, v.z), rel_ffn(D, v.y, v.z), rel_ffn(D, v.w, v.z), c, t);
}

// The FP32 form's float filter of a candidate (the first test of pair_grad): whether its float distance is below
// dhat (1 + 1e-4), i.e. whether pair_grad goes on to the float-float geometry.
__device__ inline bool pair_passes_filter(const Dev<float> &D, int ci)
{
    const int4 q = ldcg4(D.cand + ci);
    const bool ee = q.x < 0;
    const int4 v = make_int4(ee ? -1 - q.x : q.x, q.y, q.z, q.w);
    float c[4];
    v3<float> t;
    return pair_geom_ff(D, ee, v, c, t) < float(D.dhat) * 1.0001f;
}

// Barrier gradient and diagonal of one candidate (Eqs. 8-11) when d < dhat; records the pair for p^T H p.
template <typename R>
__device__ inline void pair_grad(const Dev<R> &D, int ci, int par)
{
    const int4 q = ldcg4(D.cand + ci);
    const bool ee = q.x < 0;
    int4 v = make_int4(ee ? -1 - q.x : q.x, q.y, q.z, q.w);
    R c[4];
    v3<R> t;
    R d;
    if constexpr (sizeof(R) == 4) {
        d = pair_geom_ff(D, ee, v, c, t);
        if (!(d < R(D.dhat) * R(1.0001))) return;   // float filter; the exact cut-off test follows
    } else {
        d = pair_geom<R>(ee, ldcg4(D.x + v.x), ldcg4(D.x + v.y), ldcg4(D.x + v.z), ldcg4(D.x + v.w), c, t);
        if (!(d < R(D.dhat))) return;
    }
    R A, B;
    R r = d - R(D.dhat);   // d - dhat: from the float-float distance in the FP32 form
    if constexpr (sizeof(R) == 4) {
        if (!(d < R(1e-3) * R(D.dhat))) {
            ffn cf[4];
            v3<ffn> tf;
            const ffn df = pair_geom_ffn(D, ee, v, cf, tf);
            const ffn rf = df - ffn(D.dhat);
            if (!(rf.h < 0.0f)) return;
#pragma unroll
            for (int k = 0; k < 4; ++k) c[k] = __fadd_rn(cf[k].h, cf[k].l);
            t = mkv(__fadd_rn(tf.x.h, tf.x.l), __fadd_rn(tf.y.h, tf.y.l), __fadd_rn(tf.z.h, tf.z.l));
            d = __fadd_rn(df.h, df.l);
            r = __fadd_rn(rf.h, rf.l);
        }
    }
    if (sizeof(R) == 4 && d < R(1e-3) * R(D.dhat)) {
        // near-zero distance: evaluate in double and round the results
        double cd[4];
        v3<double> td;
        double dd = pair_geom<double>(ee, ldcg4(D.x + v.x), ldcg4(D.x + v.y), ldcg4(D.x + v.z), ldcg4(D.x + v.w), cd, td);
        if (!(dd > 0.0)) { flag_error(D.ctrl, ERR_PENETRATION); return; }
        atomicAdd(&D.ctrl->n_near64, 1);
        double b1, b2;
        barrier_d12<double>(dd, D.dhat, b1, b2);
        A = R(D.kappa * (b2 / (dd * dd) - b1 / (dd * dd * dd)));
        B = R(D.kappa * b1 / dd);
        for (int k = 0; k < 4; ++k) c[k] = R(cd[k]);
        t = mkv(R(td.x), R(td.y), R(td.z));
        d = R(dd);
    } else {
        if (!(d > R(0))) { flag_error(D.ctrl, ERR_PENETRATION); return; }
        R b1, b2;
        barrier_d12r<R>(d, r, R(D.dhat), b1, b2);
        A = R(D.kappa) * (b2 / (d * d) - b1 / (d * d * d));
        B = R(D.kappa) * b1 / d;
    }
    const int slot = atomicAdd(&D.ctrl->n_active, 1);
    if (slot >= D.cand_cap) { flag_error(D.ctrl, ERR_CAPACITY); return; }
    Active<R> ap;
    ap.v = v;
#pragma unroll
    for (int k = 0; k < 4; ++k) ap.c[k] = c[k];
    ap.t[0] = t.x; ap.t[1] = t.y; ap.t[2] = t.z;
    ap.A = A; ap.B = B; ap.d = d;
    ap.ty = ee ? 1 : 0;
    D.act[slot] = ap;
    const int vid[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const R ck = c[k];
        const R ctx = ck * t.x, cty = ck * t.y, ctz = ck * t.z;
        atomic_add4<R>(&D.g[par][vid[k]], B * ctx, B * cty, B * ctz);
        const R bc = B * ck * ck;
        atomic_add4<R>(&D.dg[par][vid[k]], A * ctx * ctx + bc, A * cty * cty + bc, A * ctz * ctz + bc);
    }
}

// Gradient pass: blocks [0, ntb) own tets, the rest loop over the candidates.
template <typename R, bool CO = false>
__global__ void __launch_bounds__(EB) k_grad(Dev<R> D, int par, int ntb)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl *c = D.ctrl;
        c->rebuild = 0;
        if (c->n_cand > D.cand_cap) flag_error(c, ERR_CAPACITY);
    }
    if ((int)blockIdx.x < ntb) {
        __shared__ R sacc[6 * SCATTER_MAXU];
        tet_grad_chunk<R, CO>(D, blockIdx.x, par, sacc);
    } else {
        const int nc = min(D.ctrl->n_cand, D.cand_cap);
        const int stride = (gridDim.x - ntb) * blockDim.x;
        for (int ci = (blockIdx.x - ntb) * blockDim.x + threadIdx.x; ci < nc; ci += stride) pair_grad<R>(D, ci, par);
    }
}

// Segmented form: per-vertex gather of the (tet, corner) contributions in CSR order (deterministic).
template <typename R>
__global__ void __launch_bounds__(VB) k_gather(Dev<R> D, int par)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.nv) return;
    const int n4 = 4 * D.nt;
    R s[6] = {0, 0, 0, 0, 0, 0};
    for (int q = D.v2c_off[i]; q < D.v2c_off[i + 1]; ++q) {
        const int c = D.v2c[q];
#pragma unroll
        for (int k = 0; k < 6; ++k) s[k] += D.contrib[k * n4 + c];
    }
    typename V4<R>::T G = D.g[par][i], Dg = D.dg[par][i];
    G.x += s[0]; G.y += s[1]; G.z += s[2];
    Dg.x += s[3]; Dg.y += s[4]; Dg.z += s[5];
    D.g[par][i] = G;
    D.dg[par][i] = Dg;
}

// ------------------------------------------------------------------------------------------ a4: beta reductions

// Preconditioner entry of a free vertex of mass m (Sec. 4.2): the Jacobi entry 1/diag wherever diag > 1e-3 m, the
// inertia diagonal 1/m elsewhere.  The barrier term (b'/d) c_i^2 of Eq. 9-10 is negative inside dhat, so the
// tangential entries of a contact vertex can reach zero or go negative, where 1/diag is unbounded or negative.
template <typename R> __device__ inline R precond(R d, R m) { return R(1) / (d > R(1e-3) * m ? d : m); }

__device__ inline float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ inline double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// p_{k+1} = -P g + beta p_k of vertex i (Algorithm 1) from the stored P g (pg) and p_k; the persistent form
// evaluates it wherever a vertex's direction is needed, with one rounding order, so every evaluation agrees
// bitwise.  Kinematic vertices have pg = p = 0.
template <typename R>
__device__ inline typename V4<R>::T dir_from(const typename V4<R>::T &g, const typename V4<R>::T &p, R b, bool nzb)
{
    if (!nzb) return mk4<R>(-g.x, -g.y, -g.z, R(0));
    return mk4<R>(fma_rn(b, p.x, -g.x), fma_rn(b, p.y, -g.y), fma_rn(b, p.z, -g.z), R(0));
}
template <typename R> __device__ inline typename V4<R>::T dir_of(const Dev<R> &D, int i, R b, bool nzb)
{
    const typename V4<R>::T g = ldcg4(D.pg + i);
    if (!nzb) return dir_from<R>(g, g, b, nzb);
    return dir_from<R>(g, ldcg4(D.p + i), b, nzb);
}

// adds a b to the float-float (h, l) exactly up to the final rounding of l: FMA TwoProd, then TwoSum of the head
__device__ inline void ff_add_prod(float &h, float &l, float a, float b)
{
    const float p = __fmul_rn(a, b), e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(h, p), bp = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    h = s;
    l = __fadd_rn(l, __fadd_rn(err, e));
}
// adds a b c the same way (a b formed exactly first, its tail times c added to l)
__device__ inline void ff_add_prod3(float &h, float &l, float a, float b, float c)
{
    const float p = __fmul_rn(a, b), e = __fmaf_rn(a, b, -p);
    ff_add_prod(h, l, p, c);
    l = __fmaf_rn(e, c, l);
}

// The beta pass's sums for one vertex (Sec. 4.1-4.2) -- PR+: {g P y, g P g, g . p0}; DK: {g P y, y P y, y . p0,
// p0 . g, g P g}, with y = g - g0 -- as heads th and tails tl, and its preconditioned gradient P g.  In the FP32 form
// every product is formed exactly (FMA TwoProd) and summed in float-float: the PR and DK numerators cancel, and
// rounded float products carried about 1e-5 of beta into the direction.  m is the vertex mass (Jacobi floor).
template <typename R>
__device__ inline void beta_terms(const R gv[3], const R dv[3], const R g0[3], const R p0[3], R m, int rule, R th[5],
                                  R tl[5], R pg[3])
{
#pragma unroll
    for (int q = 0; q < 5; ++q) { th[q] = R(0); tl[q] = R(0); }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R P = precond<R>(dv[a], m);
        const R g = gv[a], y = g - g0[a];
        pg[a] = g * P;
        if constexpr (sizeof(R) == 4) {
            if (rule == 0) {
                ff_add_prod3(th[0], tl[0], g, P, y); ff_add_prod3(th[1], tl[1], g, P, g); ff_add_prod(th[2], tl[2], g, p0[a]);
            } else {
                ff_add_prod3(th[0], tl[0], g, P, y); ff_add_prod3(th[1], tl[1], y, P, y); ff_add_prod(th[2], tl[2], y, p0[a]);
                ff_add_prod(th[3], tl[3], p0[a], g); ff_add_prod3(th[4], tl[4], g, P, g);
            }
        } else {
            if (rule == 0) {
                th[0] += pg[a] * y; th[1] += pg[a] * g; th[2] += g * p0[a];
            } else {
                th[0] += pg[a] * y; th[1] += y * P * y; th[2] += y * p0[a]; th[3] += p0[a] * g; th[4] += pg[a] * g;
            }
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(VB) k_dots(Dev<R> D, int par)
{
    __shared__ double sh[32 * 5];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // PR+: {g P (g - g0), g P g, g . p0, 0, 0};  DK: {g P y, y P y, y . p0, p0 . g, g P g}
    R s[5] = {0, 0, 0, 0, 0}, sl[5] = {0, 0, 0, 0, 0};
    if (i < D.nv) {
        const typename V4<R>::T G = ldcg4(D.g[par] + i), Dg = ldcg4(D.dg[par] + i), G0 = ldcg4(D.g[par ^ 1] + i), P0 = ldcg4(D.p + i);
        if (Dg.w > R(0)) {
            const R gv[3] = {G.x, G.y, G.z}, dv[3] = {Dg.x, Dg.y, Dg.z}, g0[3] = {G0.x, G0.y, G0.z}, p0[3] = {P0.x, P0.y, P0.z};
            R pg[3];
            beta_terms<R>(gv, dv, g0, p0, Dg.w, D.beta_rule, s, sl, pg);
        }
    }
    double sd[5];
    block_sum_acc<5>(s, sl, sd, sh);
    if (publish_partials<5>(sd, D.part, &D.ctrl->ticket[TK_DOTS])) {
        double t[5];
        finish_sums<5>(t, D.part, sh);
        if (threadIdx.x == 0) {
            Ctrl *c = D.ctrl;
            double beta = 0.0, gPg, gp_new;
            int rs = 0;
            if (D.beta_rule == 0) {
                gPg = t[1];
                if (c->k > 0) {
                    beta = c->gPg_prev > 0.0 ? t[0] / c->gPg_prev : 0.0;
                    if (beta < 0.0) beta = 0.0;
                }
                gp_new = -gPg + beta * t[2];
            } else {
                gPg = t[4];
                if (c->k > 0) beta = fabs(t[2]) < 1e-30 ? 0.0 : t[0] / t[2] - (t[1] / t[2]) * (t[3] / t[2]);
                gp_new = -gPg + beta * t[3];
            }
            if (gp_new >= 0.0 && beta != 0.0) { beta = 0.0; rs = 1; }
            c->beta = beta;
            c->restarted = rs;
            c->gPg_prev = gPg;
        }
    }
}

// ------------------------------------------------------------------------------------------ a5: direction

template <typename R>
__global__ void __launch_bounds__(VB) k_dir(Dev<R> D, int par)
{
    __shared__ double sh[32 * 2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double beta = D.ctrl->beta;
    R s[2] = {0, 0};   // g . p, p^T M p + plane part
    R pm = 0;
    if (i < D.nv) {
        const typename V4<R>::T G = ldcg4(D.g[par] + i), Dg = ldcg4(D.dg[par] + i);
        typename V4<R>::T Pn = mk4<R>(R(0), R(0), R(0), R(0));
        if (Dg.w > R(0)) {
            const typename V4<R>::T P0 = ldcg4(D.p + i);
            const R b = R(beta);
            if (beta != 0.0) {
                Pn.x = -precond<R>(Dg.x, Dg.w) * G.x + b * P0.x;
                Pn.y = -precond<R>(Dg.y, Dg.w) * G.y + b * P0.y;
                Pn.z = -precond<R>(Dg.z, Dg.w) * G.z + b * P0.z;
            } else {
                Pn.x = -precond<R>(Dg.x, Dg.w) * G.x;
                Pn.y = -precond<R>(Dg.y, Dg.w) * G.y;
                Pn.z = -precond<R>(Dg.z, Dg.w) * G.z;
            }
            const R px = Pn.x, py = Pn.y, pz = Pn.z;
            s[0] = G.x * px + G.y * py + G.z * pz;
            s[1] = Dg.w * (px * px + py * py + pz * pz);
            if (D.has_plane && G.w != R(0)) {
                const R np = R(D.pn[0]) * px + R(D.pn[1]) * py + R(D.pn[2]) * pz;
                s[1] += G.w * np * np;
            }
            if (D.pnorm == 0) pm = sqrt(px * px + py * py + pz * pz);
            else pm = fmax(fabs(px), fmax(fabs(py), fabs(pz)));
        }
        D.p[i] = Pn;
    }
    double sd[2];
    block_sum_acc<2>(s, sd, sh);
    double mx;
    if constexpr (sizeof(R) == 4) mx = (double)block_max_f(pm, (float *)sh);
    else mx = block_max(pm, sh);
    double v[3] = {sd[0], sd[1], mx};
    if (publish_partials<3>(v, D.part, &D.ctrl->ticket[TK_DIR])) {
        double t[2];
        {
            const int nblk = gridDim.x;
            for (int q = 0; q < 2; ++q) {
                double a = 0.0;
                for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += __ldcg(D.part + q * nblk + b);
                t[q] = a;
            }
            block_sum<2>(t, sh);
        }
        double m = finish_max(D.part, 2, sh);
        if (threadIdx.x == 0) {
            D.ctrl->gp = t[0];
            D.ctrl->pHp_vert = t[1];
            D.ctrl->pmax = m;
        }
    }
}

// ------------------------------------------------------------------------------------------ a6-a7: p^T H p, step

// h^2 V [2 Psi_2 |dF|^2 + Psi_33 (cof(F) : dF)^2 + Psi_3 d2det(F)[dF, dF] + Psi_1 d2I1(F)[dF, dF]] (Sec. 3.1 with
// H2 = 2I, H3 the det Hessian, H1 the Hessian of tr(S)) for the direction values P0..P3 of the tet's vertices.
template <typename R, bool CO = false>
__device__ inline R tet_pHp_vec(const Dev<R> &D, int e, const int4 &tv, const typename V4<R>::T &P0,
                                const typename V4<R>::T &P1, const typename V4<R>::T &P2, const typename V4<R>::T &P3)
{
    TetF<R> T;
    tet_F<R>(D, e, tv, T);
    if (!(T.J > R(0))) { flag_error(D.ctrl, ERR_INVERTED); return R(0); }
    R dp[3][3];
    dp[0][0] = P1.x - P0.x; dp[1][0] = P1.y - P0.y; dp[2][0] = P1.z - P0.z;
    dp[0][1] = P2.x - P0.x; dp[1][1] = P2.y - P0.y; dp[2][1] = P2.z - P0.z;
    dp[0][2] = P3.x - P0.x; dp[1][2] = P3.y - P0.y; dp[2][2] = P3.z - P0.z;
    R dF[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) dF[a][b] = dp[a][0] * T.w[0][b] + dp[a][1] * T.w[1][b] + dp[a][2] * T.w[2][b];
    if constexpr (sizeof(R) == 4) {
        // FP32 form: the second derivative along dF of Psi written in C = F^T F,
        //   S : dF^T dF + k1 (tr C^-1 E)^2 + k2 tr(C^-1 E C^-1 E),   E = dF^T F + F^T dF,
        // with S = 2 dPsi/dC, C^-1, k1 = J (Psi_33 J + Psi_3) / 4, k2 = -Psi_3 J / 2 from the gradient pass at
        // the same x (formed there from the metric change, accurate for small strains).  A direction that rotates
        // the tet cancels inside E, so the large terms mu |dF|^2 and Psi_3 d2det(F)[dF, dF] of the I2/I3 form,
        // which cancel for it, never meet in float.
        const size_t n = (size_t)D.nt;
        const float4 q0 = __ldcg(D.tS + e), q1 = __ldcg(D.tS + n + e), q2 = __ldcg(D.tS + 2 * n + e);
        const float4 q3 = __ldcg(D.tS + 3 * n + e);
        if (CO && (D.model == MAT_FCR || D.model == MAT_ARAP)) {
            CorotPIn ci;
            const float rq[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w,
                                  q3.x, q3.y, q3.z, q3.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) ci.rec[k] = rq[k];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) { ci.dF[a][b] = dF[a][b]; ci.F[a][b] = T.F[a][b]; ci.cf[a][b] = T.cf[a][b]; }
            R mu, lam;
            tet_material<R>(D, e, mu, lam);
            ci.mu = mu; ci.lam = lam; ci.fcr = D.model == MAT_FCR;
            return D.hv[e] * corot_pHp(ci);
        }
        const float S00 = q0.x, S01 = q0.y, S02 = q0.z, S11 = q0.w, S12 = q1.x, S22 = q1.y;
        const float C00 = q1.z, C01 = q1.w, C02 = q2.x, C11 = q2.y, C12 = q2.z, C22 = q2.w;
        const float k1 = q3.x, k2 = q3.y;
        float E[3][3], DD[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
                float fe = 0.0f, dd = 0.0f;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    fe += dF[r][a] * T.F[r][b] + T.F[r][a] * dF[r][b];
                    dd += dF[r][a] * dF[r][b];
                }
                E[a][b] = E[b][a] = fe;
                DD[a][b] = DD[b][a] = dd;
            }
        const float Ci[3][3] = {{C00, C01, C02}, {C01, C11, C12}, {C02, C12, C22}};
        float X[3][3];   // C^-1 E
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) X[a][b] = Ci[a][0] * E[0][b] + Ci[a][1] * E[1][b] + Ci[a][2] * E[2][b];
        const float trX = X[0][0] + X[1][1] + X[2][2];
        float trX2 = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) trX2 += X[a][b] * X[b][a];
        const float SD = S00 * DD[0][0] + S11 * DD[1][1] + S22 * DD[2][2] +
                         2.0f * (S01 * DD[0][1] + S02 * DD[0][2] + S12 * DD[1][2]);
        return D.hv[e] * (SD + k1 * trX * trX + k2 * trX2);
    }
    R mu, lam;
    tet_material<R>(D, e, mu, lam);
    const MatTerms<R> mt = mat_terms<R>(D.model, mu, lam, T.J);
    R n2 = 0, g3 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) { n2 += dF[a][b] * dF[a][b]; g3 += T.cf[a][b] * dF[a][b]; }
    // columns: f_b = F[.][b], df_b = dF[.][b]
    v3<R> f0 = mkv(T.F[0][0], T.F[1][0], T.F[2][0]), f1 = mkv(T.F[0][1], T.F[1][1], T.F[2][1]),
          f2 = mkv(T.F[0][2], T.F[1][2], T.F[2][2]);
    v3<R> d0 = mkv(dF[0][0], dF[1][0], dF[2][0]), d1 = mkv(dF[0][1], dF[1][1], dF[2][1]),
          d2 = mkv(dF[0][2], dF[1][2], dF[2][2]);
    const R h3 = R(2) * (dot(d0, cross(d1, f2)) + dot(d0, cross(f1, d2)) + dot(f0, cross(d1, d2)));
    R q = mt.c2 * n2 + mt.Psi33 * g3 * g3 + mt.Psi3 * h3;
    if constexpr (sizeof(R) == 8) {
        if (mt.Psi1 != R(0)) {
            Polar pol;
            polar_of(T.F, pol);
            q += mt.Psi1 * polar_h1(pol, dF);
        }
    }
    return D.hv[e] * q;
}

template <typename R, bool CO = false>
__device__ inline R tet_pHp(const Dev<R> &D, int e)
{
    const int4 tv = D.tet[e];
    return tet_pHp_vec<R, CO>(D, e, tv, ldcg4(D.p + tv.x), ldcg4(D.p + tv.y), ldcg4(D.p + tv.z), ldcg4(D.p + tv.w));
}

// Eqs. 12-13 with the recorded A = kappa (b''/d^2 - b'/d^3), B = kappa b'/d, for direction values P0..P3, in
// double: B = kappa b'/d is negative, so the two terms cancel in part (pairs are few)
template <typename R>
__device__ inline void load_active(const Dev<R> &D, int k, Active<R> &ap)
{
    const int4 *src = reinterpret_cast<const int4 *>(D.act + k);
    int4 *dst = reinterpret_cast<int4 *>(&ap);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(Active<R>) / sizeof(int4)); ++w) dst[w] = __ldcg(src + w);
}
template <typename R>
__device__ inline double pair_pHp_vec(const Active<R> &ap, const typename V4<R>::T &P0, const typename V4<R>::T &P1,
                                      const typename V4<R>::T &P2, const typename V4<R>::T &P3)
{
    // sum c_i p_i is the relative motion of the pair (sum c_i = 0): it cancels when the pair moves together, so it
    // is formed in double (the products of two floats are exact there)
    const double c0 = ap.c[0], c1 = ap.c[1], c2 = ap.c[2], c3 = ap.c[3];
    const double cx = c0 * double(P0.x) + c1 * double(P1.x) + c2 * double(P2.x) + c3 * double(P3.x);
    const double cy = c0 * double(P0.y) + c1 * double(P1.y) + c2 * double(P2.y) + c3 * double(P3.y);
    const double cz = c0 * double(P0.z) + c1 * double(P1.z) + c2 * double(P2.z) + c3 * double(P3.z);
    const double ct = cx * double(ap.t[0]) + cy * double(ap.t[1]) + cz * double(ap.t[2]);
    return double(ap.A) * ct * ct + double(ap.B) * (cx * cx + cy * cy + cz * cz);
}
template <typename R>
__device__ inline double pair_pHp(const Dev<R> &D, int k)
{
    Active<R> ap;
    load_active<R>(D, k, ap);
    return pair_pHp_vec<R>(ap, ldcg4(D.p + ap.v.x), ldcg4(D.p + ap.v.y), ldcg4(D.p + ap.v.z), ldcg4(D.p + ap.v.w));
}

// The step rule of Sec. 4.3 and the predicted decrease of Sec. 4.4, in the last block of k_pHp.
template <typename R>
__device__ inline void finish_step(const Dev<R> &D, double pHp)
{
    Ctrl *c = D.ctrl;
    const double gp = c->gp, pmax = c->pmax;
    const double au = pmax > 0.0 ? D.dhat / (2.0 * pmax) : 0.0;
    const double ab = -gp / pHp;
    double a;
    int capped;
    if (!(pHp > 0.0) || !isfinite(ab)) { a = au; capped = 1; }
    else if (ab < au) { a = ab; capped = 0; }
    else { a = au; capped = 1; }
    const double dE = -a * gp - 0.5 * a * a * pHp;
    const int k = c->k;
    if (!isfinite(a) || !isfinite(gp)) flag_error(c, ERR_NONFINITE);
    if (c->err != 0u || c->converged) a = 0.0;
    c->pHp = pHp; c->alpha_bar = ab; c->alpha_up = au; c->alpha = a; c->dE = dE; c->capped = capped;
    c->n_active_last = c->n_active;
    if (!c->converged && c->err == 0u) {
        if (k == 0) c->dE0 = dE;
        c->n_capped += capped;
        c->iters_done = k + 1;
        if (D.trace && k < D.iters) {
            double *tr = D.trace + (size_t)k * TRACE_COLS;
            tr[0] = c->beta; tr[1] = gp; tr[2] = pHp; tr[3] = pmax; tr[4] = a; tr[5] = dE;
            tr[6] = c->n_active; tr[7] = capped;
        }
        if (D.eps > 0.0 && dE < D.eps * c->dE0) c->converged = 1;
    }
    c->k = k + 1;
}

template <typename R, bool CO = false>
__global__ void __launch_bounds__(EB) k_pHp(Dev<R> D, int ntb)
{
    __shared__ double sh[32];
    double sd[1] = {0.0};
    if ((int)blockIdx.x < ntb) {
        R s[1] = {R(0)};
        const int e = blockIdx.x * blockDim.x + threadIdx.x;
        if (e < D.nt) s[0] = tet_pHp<R, CO>(D, e);
        block_sum_acc<1>(s, sd, sh);
    } else {
        const int na = D.ctrl->n_active;
        const int stride = (gridDim.x - ntb) * blockDim.x;
        for (int k = (blockIdx.x - ntb) * blockDim.x + threadIdx.x; k < na; k += stride) sd[0] += pair_pHp<R>(D, k);
        block_sum<1>(sd, sh);
    }
    if (publish_partials<1>(sd, D.part, &D.ctrl->ticket[TK_PHP])) {
        double t[1];
        finish_sums<1>(t, D.part, sh);
        if (threadIdx.x == 0) finish_step<R>(D, t[0] + D.ctrl->pHp_vert);
    }
}

// ------------------------------------------------------------------------------------------ a8: update

// x += alpha p, then the inertia / plane initialisation of the next iteration's accumulators (parity par ^ 1) and
// the displacement check for the candidate padding.
template <typename R>
__global__ void __launch_bounds__(VB) k_update(Dev<R> D, int par)
{
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double a = D.ctrl->alpha;
    double md2 = 0.0;
    if (i < D.nv) {
        const typename V4<R>::T P = ldcg4(D.p + i);
        double4_32a X = ldcg4(D.x + i);
        if constexpr (sizeof(R) == 4) {
            const ffl as = ff_split(a);
            const float4 xh = update_vertex<R>(D, i, X, P, a, as.h, as.l, X, par ^ 1);
            const float4 b = D.xbh[i];
            const float x = xh.x - b.x, y = xh.y - b.y, z = xh.z - b.z;
            md2 = (double)(x * x + y * y + z * z);
        } else {
            update_vertex<R>(D, i, X, P, a, 0.0f, 0.0f, ldcg4(D.xtil + i), par ^ 1);
            md2 = disp2<R>(D, i, X);
        }
    }
    double mx = block_max(md2, sh);
    double v1[1] = {mx};
    if (publish_partials<1>(v1, D.part, &D.ctrl->ticket[TK_UPDATE])) {
        double m = finish_max(D.part, 0, sh);
        if (threadIdx.x == 0) {
            D.ctrl->n_active = 0;
            request_rebuild_if(D, m);
        }
    }
}

// v = (x - x^t) / h; on a kernel error the step is undone (x = x^t) and the velocity kept.
template <typename R>
__global__ void __launch_bounds__(VB) k_finish(Dev<R> D)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = D.ctrl->err != 0u;
    if (i < D.nv) {
        const double4_32a X = D.x[i], XT = D.xt[i];
        if (bad) {
            put_x<R>(D, i, XT);
        } else {
            const double ih = 1.0 / D.h;
            double4_32a V = D.v[i];
            V.x = (X.x - XT.x) * ih; V.y = (X.y - XT.y) * ih; V.z = (X.z - XT.z) * ih;
            D.v[i] = V;
        }
    }
    if (i == 0) {
        if (bad) { if (D.ctrl->err_step < 0) D.ctrl->err_step = (int)D.ctrl->step; }
        else D.ctrl->step += 1;
    }
}

// ------------------------------------------------------------------------------------------ energy (reporting)

template <typename R>
__global__ void __launch_bounds__(EB) k_energy(Dev<R> D, int ntb, int nvb)
{
    __shared__ double sh[32 * 4];
    double s[4] = {0, 0, 0, 0};
    const int b = blockIdx.x;
    if (b < ntb) {
        const int e = b * blockDim.x + threadIdx.x;
        if (e < D.nt) {
            const int4 tv = D.tet[e];
            TetF<double> T;
            // energy is evaluated in double in both forms
            double ds[3][3];
            const double4_32a X0 = D.x[tv.x], X1 = D.x[tv.y], X2 = D.x[tv.z], X3 = D.x[tv.w];
            ds[0][0] = X1.x - X0.x; ds[1][0] = X1.y - X0.y; ds[2][0] = X1.z - X0.z;
            ds[0][1] = X2.x - X0.x; ds[1][1] = X2.y - X0.y; ds[2][1] = X2.z - X0.z;
            ds[0][2] = X3.x - X0.x; ds[1][2] = X3.y - X0.y; ds[2][2] = X3.z - X0.z;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) T.w[r][c] = double(D.Dm[(3 * r + c) * D.nt + e]);
            double I2 = 0;
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    T.F[a][c] = ds[a][0] * T.w[0][c] + ds[a][1] * T.w[1][c] + ds[a][2] * T.w[2][c];
                    I2 += T.F[a][c] * T.F[a][c];
                }
            const double J = T.F[0][0] * (T.F[1][1] * T.F[2][2] - T.F[2][1] * T.F[1][2]) -
                             T.F[0][1] * (T.F[1][0] * T.F[2][2] - T.F[2][0] * T.F[1][2]) +
                             T.F[0][2] * (T.F[1][0] * T.F[2][1] - T.F[2][0] * T.F[1][1]);
            if (!(J > 0.0)) flag_error(D.ctrl, ERR_INVERTED);
            else {
                double mu = D.mu, lam = D.lam;
                if (D.escale) { mu *= D.escale[e]; lam *= D.escale[e]; }
                double I1 = 3.0;
                if (D.model == MAT_FCR || D.model == MAT_ARAP) {
                    Polar pol;
                    polar_of(T.F, pol);
                    I1 = pol.trS;
                }
                s[1] = double(D.hv[e]) * mat_psi(D.model, mu, lam, I1, I2, J);
            }
        }
    } else if (b < ntb + nvb) {
        const int i = (b - ntb) * blockDim.x + threadIdx.x;
        if (i < D.nv) {
            const double4_32a X = D.x[i], XT = D.xtil[i];
            const double m = XT.w > 0.0 ? XT.w : 0.0;
            s[0] = 0.5 * m * dist2(X, XT);
            if (D.has_plane) {
                double d = D.pn[0] * X.x + D.pn[1] * X.y + D.pn[2] * X.z - D.po;
                if (d < D.dhat) {
                    if (!(d > 0.0)) flag_error(D.ctrl, ERR_PENETRATION);
                    else s[3] = D.kappa * barrier_b<double>(d, D.dhat);
                }
            }
        }
    } else {
        const int nc = min(D.ctrl->n_cand, D.cand_cap);
        const int stride = (gridDim.x - ntb - nvb) * blockDim.x;
        for (int ci = (b - ntb - nvb) * blockDim.x + threadIdx.x; ci < nc; ci += stride) {
            const int4 q = D.cand[ci];
            const bool ee = q.x < 0;
            const double4_32a X0 = D.x[ee ? -1 - q.x : q.x], X1 = D.x[q.y], X2 = D.x[q.z], X3 = D.x[q.w];
            double c[4];
            v3<double> t;
            const double d = pair_geom<double>(ee, X0, X1, X2, X3, c, t);
            if (d < D.dhat) {
                if (!(d > 0.0)) flag_error(D.ctrl, ERR_PENETRATION);
                else s[2] += D.kappa * barrier_b<double>(d, D.dhat);
            }
        }
    }
    block_sum<4>(s, sh);
    if (publish_partials<4>(s, D.part, &D.ctrl->ticket[TK_ENERGY])) {
        double t[4];
        finish_sums<4>(t, D.part, sh);
        if (threadIdx.x == 0)
            for (int q = 0; q < 4; ++q) D.ctrl->energy[q] = t[q];
    }
}

} // namespace pncg
