// Differentiation of a simulated trajectory by the adjoint method.  Each time step is taken as the solution of
// grad E(x_{t+1}; x~_t, theta) = 0 (Algorithm 1's minimisation), x~_t = x_t + h v_t + h^2 g, v_{t+1} = (x_{t+1} - x_t)/h.
// The implicit function theorem gives H dx_{t+1} = M dx~_t - (d grad E / d theta) d theta with H the Hessian of E at
// x_{t+1} (inertia, elastic density, barrier with the closest points frozen as in Sec. 3.2, half-space barrier), so a
// reverse step solves H lambda = abar_x(t+1) + abar_v(t+1)/h and carries abar_x~ = M lambda back:
//   abar_x(t) = M lambda - abar_v(t+1)/h,   abar_v(t) = h M lambda,   abar_E_e -= lambda_e . d g_e / d E_e.
// H is applied matrix-free (the vector form of the p^T H p terms); the solve is Jacobi-preconditioned linear CG with
// the preconditioner of Sec. 4.2.  Kinematic vertices: rows and columns of H dropped, lambda = 0 there.
#pragma once

#include "kernels.cuh"

namespace pncg {

// Hessian times v, vertex part (inertia and half-space barrier; kinematic rows zero): written, not added.
// Needs the gradient pass at x (dg.w = mass or -1, g.w = kappa b'' of the half-space).
template <typename R>
__global__ void k_hvp_vert(Dev<R> D, int par, const double *v, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.nv) return;
    const typename V4<R>::T G = D.g[par][i], Dg = D.dg[par][i];
    double o[3] = {0.0, 0.0, 0.0};
    if (Dg.w > R(0)) {
        const double m = Dg.w;
        const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
        o[0] = m * vx; o[1] = m * vy; o[2] = m * vz;
        if (D.has_plane && G.w != R(0)) {
            const double nv = D.pn[0] * vx + D.pn[1] * vy + D.pn[2] * vz, k = double(G.w) * nv;
            o[0] += k * D.pn[0]; o[1] += k * D.pn[1]; o[2] += k * D.pn[2];
        }
    }
    out[3 * i] = o[0]; out[3 * i + 1] = o[1]; out[3 * i + 2] = o[2];
}

template <typename R> __device__ inline v3<R> vload(const Dev<R> &D, const double *v, int i)
{
    // kinematic columns of H are dropped: their v entries count as zero
    if (D.xtil[i].w < 0.0) return mkv(R(0), R(0), R(0));
    return mkv(R(v[3 * i]), R(v[3 * i + 1]), R(v[3 * i + 2]));
}
template <typename R> __device__ inline void vadd(const Dev<R> &D, double *out, int i, R a, R b, R c)
{
    if (D.xtil[i].w < 0.0) return;
    atomicAdd(out + 3 * i, double(a));
    atomicAdd(out + 3 * i + 1, double(b));
    atomicAdd(out + 3 * i + 2, double(c));
}

// Elastic tet part: h^2 V dP(dF) W^T scattered to the corners, dP = 2 Psi_2 dF + Psi_33 (cof F : dF) cof F +
// Psi_3 d cof(F)[dF] + Psi_1 H1[dF] (the differential of P = Psi_1 R + 2 Psi_2 F + Psi_3 cof F; the I1 term of the
// fixed corotated and as-rigid-as-possible densities from the polar decomposition, in double); p^T (H v) equals the
// p^T H p form of Sec. 3.1.
template <typename R>
__global__ void __launch_bounds__(EB) k_hvp_tet(Dev<R> D, const double *v, double *out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D.nt) return;
    const int4 tv = D.tet[e];
    TetF<R> T;
    tet_F<R>(D, e, tv, T);
    if (!(T.J > R(0))) { flag_error(D.ctrl, ERR_INVERTED); return; }
    const v3<R> V0 = vload(D, v, tv.x), V1 = vload(D, v, tv.y), V2 = vload(D, v, tv.z), V3 = vload(D, v, tv.w);
    R dp[3][3];
    dp[0][0] = V1.x - V0.x; dp[1][0] = V1.y - V0.y; dp[2][0] = V1.z - V0.z;
    dp[0][1] = V2.x - V0.x; dp[1][1] = V2.y - V0.y; dp[2][1] = V2.z - V0.z;
    dp[0][2] = V3.x - V0.x; dp[1][2] = V3.y - V0.y; dp[2][2] = V3.z - V0.z;
    R dF[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) dF[a][b] = dp[a][0] * T.w[0][b] + dp[a][1] * T.w[1][b] + dp[a][2] * T.w[2][b];
    R mu, lam;
    tet_material<R>(D, e, mu, lam);
    const MatTerms<R> mt = mat_terms<R>(D.model, mu, lam, T.J);
    R g3 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) g3 += T.cf[a][b] * dF[a][b];
    const v3<R> f0 = mkv(T.F[0][0], T.F[1][0], T.F[2][0]), f1 = mkv(T.F[0][1], T.F[1][1], T.F[2][1]),
                f2 = mkv(T.F[0][2], T.F[1][2], T.F[2][2]);
    const v3<R> d0 = mkv(dF[0][0], dF[1][0], dF[2][0]), d1 = mkv(dF[0][1], dF[1][1], dF[2][1]),
                d2 = mkv(dF[0][2], dF[1][2], dF[2][2]);
    // columns of d cof(F)[dF]: d(f1 x f2), d(f2 x f0), d(f0 x f1)
    const v3<R> c0 = cross(d1, f2) + cross(f1, d2), c1 = cross(d2, f0) + cross(f2, d0), c2 = cross(d0, f1) + cross(f0, d1);
    const R dcof[3][3] = {{c0.x, c1.x, c2.x}, {c0.y, c1.y, c2.y}, {c0.z, c1.z, c2.z}};
    const R sc = D.hv[e];
    R dP[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) dP[a][b] = sc * (mt.c2 * dF[a][b] + mt.Psi33 * g3 * T.cf[a][b] + mt.Psi3 * dcof[a][b]);
    if (mt.Psi1 != R(0)) {
        double Fd[3][3], dFd[3][3], H1[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) { Fd[a][b] = double(T.F[a][b]); dFd[a][b] = double(dF[a][b]); }
        Polar pol;
        polar_of(Fd, pol);
        polar_h1_vec(pol, dFd, H1);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) dP[a][b] += sc * R(double(mt.Psi1) * H1[a][b]);
    }
    R o[4][3];
#pragma unroll
    for (int i = 1; i < 4; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) o[i][a] = dP[a][0] * T.w[i - 1][0] + dP[a][1] * T.w[i - 1][1] + dP[a][2] * T.w[i - 1][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) o[0][a] = -(o[1][a] + o[2][a] + o[3][a]);
    const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) vadd<R>(D, out, vid[i], o[i][0], o[i][1], o[i][2]);
}

// Barrier pair part with the closest points frozen (Eqs. 12-13 as an operator): w = sum_j c_j v_j,
// (H v)_k += c_k (A (w . t) t + B w).  In double: the pair terms cancel in part.
template <typename R>
__global__ void __launch_bounds__(EB) k_hvp_pair(Dev<R> D, const double *v, double *out)
{
    const int na = D.ctrl->n_active;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < na; k += gridDim.x * blockDim.x) {
        Active<R> ap;
        load_active<R>(D, k, ap);
        const int vid[4] = {ap.v.x, ap.v.y, ap.v.z, ap.v.w};
        double w[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const v3<R> V = vload(D, v, vid[j]);
            w[0] += double(ap.c[j]) * double(V.x); w[1] += double(ap.c[j]) * double(V.y); w[2] += double(ap.c[j]) * double(V.z);
        }
        const double s = w[0] * double(ap.t[0]) + w[1] * double(ap.t[1]) + w[2] * double(ap.t[2]);
        const double A = ap.A, Bc = ap.B;
        double f[3];
        for (int a = 0; a < 3; ++a) f[a] = A * s * double(ap.t[a]) + Bc * w[a];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (D.xtil[vid[j]].w < 0.0) continue;
            const double cj = ap.c[j];
            atomicAdd(out + 3 * vid[j], cj * f[0]);
            atomicAdd(out + 3 * vid[j] + 1, cj * f[1]);
            atomicAdd(out + 3 * vid[j] + 2, cj * f[2]);
        }
    }
}

// ---- linear CG on H lambda = b (Jacobi-preconditioned); scalars in cg[]: 0 r.z, 1 p.q, 2 alpha, 3 beta, 4 r.r,
// 5 b.b.  Reductions finish in the last block to arrive (block partials summed in block order).
enum { CG_RZ = 0, CG_PQ, CG_ALPHA, CG_BETA, CG_RR, CG_BB, CG_N };

template <typename R> __device__ inline double jacobi(const Dev<R> &D, int par, int i, int a)
{
    const typename V4<R>::T Dg = D.dg[par][i];
    if (!(Dg.w > R(0))) return 0.0;
    const R d = a == 0 ? Dg.x : (a == 1 ? Dg.y : Dg.z);
    return double(precond<R>(d, Dg.w));
}

// r = b (kinematic rows zero), z = P r, p = z, x = 0; cg[RZ] = r.z, cg[BB] = b.b
template <typename R>
__global__ void __launch_bounds__(VB) k_cg_init(Dev<R> D, int par, const double *b, double *x, double *r, double *z,
                                                double *p, double *cg, unsigned int *ticket)
{
    __shared__ double sh[32 * 2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s[2] = {0.0, 0.0};
    if (i < D.nv) {
        const bool free_v = D.xtil[i].w >= 0.0;
        for (int a = 0; a < 3; ++a) {
            const double ri = free_v ? b[3 * i + a] : 0.0, zi = jacobi<R>(D, par, i, a) * ri;
            r[3 * i + a] = ri; z[3 * i + a] = zi; p[3 * i + a] = zi; x[3 * i + a] = 0.0;
            s[0] += ri * zi; s[1] += ri * ri;
        }
    }
    block_sum<2>(s, sh);
    if (publish_partials<2>(s, D.part, ticket)) {
        double t[2];
        finish_sums<2>(t, D.part, sh);
        if (threadIdx.x == 0) { cg[CG_RZ] = t[0]; cg[CG_BB] = t[1]; cg[CG_RR] = t[1]; }
    }
}

// cg[PQ] = p.q, alpha = r.z / p.q
static __global__ void __launch_bounds__(VB) k_cg_pq(int n3, const double *p, const double *q, double *part, double *cg,
                                              unsigned int *ticket)
{
    __shared__ double sh[32];
    double s[1] = {0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n3; j += gridDim.x * blockDim.x) s[0] += p[j] * q[j];
    block_sum<1>(s, sh);
    if (publish_partials<1>(s, part, ticket)) {
        double t[1];
        finish_sums<1>(t, part, sh);
        if (threadIdx.x == 0) {
            cg[CG_PQ] = t[0];
            cg[CG_ALPHA] = t[0] != 0.0 ? cg[CG_RZ] / t[0] : 0.0;
        }
    }
}

// x += alpha p, r -= alpha q, z = P r; beta = r.z_new / r.z, r.r
template <typename R>
__global__ void __launch_bounds__(VB) k_cg_update(Dev<R> D, int par, double *x, double *r, double *z, const double *p,
                                                  const double *q, double *cg, unsigned int *ticket)
{
    __shared__ double sh[32 * 2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double al = cg[CG_ALPHA];
    double s[2] = {0.0, 0.0};
    if (i < D.nv) {
        for (int a = 0; a < 3; ++a) {
            const int j = 3 * i + a;
            x[j] += al * p[j];
            const double ri = r[j] - al * q[j], zi = jacobi<R>(D, par, i, a) * ri;
            r[j] = ri; z[j] = zi;
            s[0] += ri * zi; s[1] += ri * ri;
        }
    }
    block_sum<2>(s, sh);
    if (publish_partials<2>(s, D.part, ticket)) {
        double t[2];
        finish_sums<2>(t, D.part, sh);
        if (threadIdx.x == 0) {
            cg[CG_BETA] = cg[CG_RZ] != 0.0 ? t[0] / cg[CG_RZ] : 0.0;
            cg[CG_RZ] = t[0];
            cg[CG_RR] = t[1];
        }
    }
}

// p = z + beta p
static __global__ void k_cg_dir(int n3, const double *z, double *p, const double *cg)
{
    const double bt = cg[CG_BETA];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n3; j += gridDim.x * blockDim.x) p[j] = z[j] + bt * p[j];
}

// ---- the reverse step's vertex bookkeeping
// rhs = abar_x + abar_v / h on free vertices
template <typename R>
__global__ void k_adj_rhs(Dev<R> D, const double *ax, const double *av, double *b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.nv) return;
    const bool free_v = D.xtil[i].w >= 0.0;
    for (int a = 0; a < 3; ++a) b[3 * i + a] = free_v ? ax[3 * i + a] + av[3 * i + a] / D.h : 0.0;
}
// abar_x(t) = M lambda - abar_v(t+1)/h, abar_v(t) = h M lambda (free vertices);
// kinematic: abar_x(t) = -abar_v(t+1)/h (v(t+1) = (target - x(t))/h), abar_v(t) = 0
template <typename R>
__global__ void k_adj_out(Dev<R> D, const double *lam, const double *av, double *ax_t, double *av_t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.nv) return;
    const bool free_v = D.xtil[i].w >= 0.0;
    const double m = D.mass[i];
    for (int a = 0; a < 3; ++a) {
        const double ml = free_v ? m * lam[3 * i + a] : 0.0;
        ax_t[3 * i + a] = ml - av[3 * i + a] / D.h;
        av_t[3 * i + a] = D.h * ml;
    }
}
// dE_e -= lambda_e . d g_e / d E_e: the tet's elastic gradient is linear in E_e (mu and lambda are), so its
// derivative is the gradient evaluated with E_e = 1 (D carries mu and lambda of E = 1 and no per-tet scale)
template <typename R>
__global__ void __launch_bounds__(EB) k_adj_youngs(Dev<R> D, const double *lam, double *dE)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D.nt) return;
    TetIn<R> in;
    load_tet_in<R>(D, e, in);
    R gv[4][3], dv[4][3];
    if (!tet_grad_eval<R>(D, in, gv, dv)) return;
    const int vid[4] = {in.tv.x, in.tv.y, in.tv.z, in.tv.w};
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) s += lam[3 * vid[i] + a] * double(gv[i][a]);
    dE[e] -= s;
}

} // namespace pncg
