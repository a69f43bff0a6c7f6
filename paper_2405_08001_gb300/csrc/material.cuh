// Energy densities of the invariants I1 = tr(S) (F = R S), I2 = tr(F^T F), I3 = det F (Sec. 3.1), and the terms
// of their split Hessian that the gradient, Jacobi-diagonal and p^T H p passes need:
//   NH   mu/2 (I2 - 3) - mu log I3 + lambda/2 (log I3)^2        (the paper's Neo-Hookean, the default)
//   SNH  mu/2 (I2 - 3) - mu (I3 - 1) + lambda/2 (I3 - 1)^2       (stable Neo-Hookean)
//   FCR  mu (I2 - 2 I1 + 3) + lambda/2 (I3 - 1)^2               (fixed corotated, mu |F - R|^2 + ...)
//   ARAP mu (I2 - 2 I1 + 3)                                      (as-rigid-as-possible, mu |F - R|^2)
// None has Psi_11 or Psi_22 terms, so P = Psi_1 R + 2 Psi_2 F + Psi_3 cof(F) and
//   dF : d2Psi/dF2 : dF = 2 Psi_2 |dF|^2 + Psi_33 (cof(F) : dF)^2 + Psi_3 d2det(F)[dF, dF] + Psi_1 d2I1(F)[dF, dF].
//
// The I1 terms (FCR, ARAP) need no singular value decomposition.  In the FP64 form the rotation R comes from the scaled
// Newton iteration X <- (g X + X^-T / g) / 2, g = |det X|^(-1/3) (Higham, 1986), started at F (det F > 0), and
// S = R^T F.  Differentiating F = R S with R^T dR = [w]x skew and dS symmetric gives 2 skew(R^T dF) = [(tr(S) I -
// S) w]x, so with a = axial(R^T dF - dF^T R):
//   d2I1(F)[dF, dF] = dF : dR[dF] = a^T (tr(S) I - S)^-1 a,
// and for the diagonal (dF = e_c w^T, w a vertex's weight vector, rho = R^T e_c) a = w x rho.  The FP32 form takes
// U - I = sqrt(I + (C - I)) - I from the accurate metric change by a Newton square root instead (kernels.cuh,
// corot_terms), so that the stress keeps its relative accuracy near a rotation.
#pragma once

namespace pncg {

enum { MAT_NH = 0, MAT_SNH = 1, MAT_FCR = 2, MAT_ARAP = 3 };

template <typename R> struct MatTerms {
    R c2;     // 2 Psi_2: the coefficient of F in P and of |dF|^2 in the quadratic form
    R Psi1;   // dPsi / dI1 (FCR, ARAP)
    R Psi3, Psi33;
};

// The derivatives of the density at J = det F > 0 (mu, lambda of the tet).
template <typename R> __host__ __device__ inline MatTerms<R> mat_terms(int model, R mu, R lam, R J)
{
    MatTerms<R> t;
    t.Psi1 = R(0);
    if (model == MAT_SNH) {
        t.c2 = mu;
        t.Psi3 = -mu + lam * (J - R(1));
        t.Psi33 = lam;
    } else if (model == MAT_FCR || model == MAT_ARAP) {
        t.c2 = R(2) * mu;
        t.Psi1 = R(-2) * mu;
        t.Psi3 = model == MAT_FCR ? lam * (J - R(1)) : R(0);
        t.Psi33 = model == MAT_FCR ? lam : R(0);
    } else {
        const R L = log(J);
        t.c2 = mu;
        t.Psi3 = (lam * L - mu) / J;
        t.Psi33 = (mu + lam * (R(1) - L)) / (J * J);
    }
    return t;
}

// The density itself (energy evaluation).  I1 is only read by FCR and ARAP.
__host__ __device__ inline double mat_psi(int model, double mu, double lam, double I1, double I2, double J)
{
    if (model == MAT_SNH) return 0.5 * mu * (I2 - 3.0) - mu * (J - 1.0) + 0.5 * lam * (J - 1.0) * (J - 1.0);
    if (model == MAT_FCR) return mu * (I2 - 2.0 * I1 + 3.0) + 0.5 * lam * (J - 1.0) * (J - 1.0);
    if (model == MAT_ARAP) return mu * (I2 - 2.0 * I1 + 3.0);
    const double L = log(J);
    return 0.5 * mu * (I2 - 3.0) - mu * L + 0.5 * lam * L * L;
}

// The rotation of the polar decomposition, tr(S) and the inverse of tr(S) I - S (symmetric, positive definite: its
// eigenvalues are the pairwise sums of the singular values).
struct Polar {
    double R[3][3];
    double trS;
    double Mi[3][3];
};

struct Mat33 { double m[3][3]; };

// Not inlined, arguments and result by value: the iteration's temporaries stay out of the register budget of the
// passes that call it (which also run the Neo-Hookean path).
static __device__ __noinline__ Polar polar_value(Mat33 Fm)
{
    const double (&F)[3][3] = Fm.m;
    Polar P;
    double X[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) X[a][b] = F[a][b];
    for (int it = 0; it < 12; ++it) {
        double cf[3][3];   // cofactors: X^-T = cof(X) / det X
        cf[0][0] = X[1][1] * X[2][2] - X[1][2] * X[2][1];
        cf[0][1] = X[1][2] * X[2][0] - X[1][0] * X[2][2];
        cf[0][2] = X[1][0] * X[2][1] - X[1][1] * X[2][0];
        cf[1][0] = X[2][1] * X[0][2] - X[2][2] * X[0][1];
        cf[1][1] = X[2][2] * X[0][0] - X[2][0] * X[0][2];
        cf[1][2] = X[2][0] * X[0][1] - X[2][1] * X[0][0];
        cf[2][0] = X[0][1] * X[1][2] - X[0][2] * X[1][1];
        cf[2][1] = X[0][2] * X[1][0] - X[0][0] * X[1][2];
        cf[2][2] = X[0][0] * X[1][1] - X[0][1] * X[1][0];
        const double det = X[0][0] * cf[0][0] + X[0][1] * cf[0][1] + X[0][2] * cf[0][2];
        const double g = 1.0 / cbrt(det);
        const double gi = 1.0 / (g * det);
        double ch = 0.0, nx = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double y = 0.5 * (g * X[a][b] + gi * cf[a][b]);
                ch += (y - X[a][b]) * (y - X[a][b]);
                nx += y * y;
                X[a][b] = y;
            }
        if (ch <= 1e-30 * nx) break;
    }
    double S[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            P.R[a][b] = X[a][b];
            S[a][b] = X[0][a] * F[0][b] + X[1][a] * F[1][b] + X[2][a] * F[2][b];
        }
    P.trS = S[0][0] + S[1][1] + S[2][2];
    // M = tr(S) I - S, symmetrised
    const double m00 = P.trS - S[0][0], m11 = P.trS - S[1][1], m22 = P.trS - S[2][2];
    const double m01 = -0.5 * (S[0][1] + S[1][0]), m02 = -0.5 * (S[0][2] + S[2][0]), m12 = -0.5 * (S[1][2] + S[2][1]);
    const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
    const double c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
    const double id = 1.0 / (m00 * c00 + m01 * c01 + m02 * c02);
    P.Mi[0][0] = c00 * id; P.Mi[1][1] = c11 * id; P.Mi[2][2] = c22 * id;
    P.Mi[0][1] = P.Mi[1][0] = c01 * id;
    P.Mi[0][2] = P.Mi[2][0] = c02 * id;
    P.Mi[1][2] = P.Mi[2][1] = c12 * id;
    return P;
}

__device__ inline void polar_of(const double F[3][3], Polar &P)
{
    Mat33 Fm;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Fm.m[a][b] = F[a][b];
    P = polar_value(Fm);
}

__device__ inline double quad_Mi(const Polar &P, double a0, double a1, double a2)
{
    return a0 * (P.Mi[0][0] * a0 + P.Mi[0][1] * a1 + P.Mi[0][2] * a2) +
           a1 * (P.Mi[1][0] * a0 + P.Mi[1][1] * a1 + P.Mi[1][2] * a2) +
           a2 * (P.Mi[2][0] * a0 + P.Mi[2][1] * a1 + P.Mi[2][2] * a2);
}

// d2I1(F)[dF, dF] = a^T (tr(S) I - S)^-1 a with a = axial(R^T dF - dF^T R)
__device__ inline double polar_h1(const Polar &P, const double dF[3][3])
{
    double K[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) K[a][b] = P.R[0][a] * dF[0][b] + P.R[1][a] * dF[1][b] + P.R[2][a] * dF[2][b];
    return quad_Mi(P, K[2][1] - K[1][2], K[0][2] - K[2][0], K[1][0] - K[0][1]);
}

// the operator form of polar_h1: H1[dF] = R [Mi a]x^T with a = axial(R^T dF - dF^T R), so that
// dF : H1[dF] = a^T Mi a (a . b = (R^T dF) : B(b) for the skew B(b) with B21 = b0, B02 = b1, B10 = b2)
__device__ inline void polar_h1_vec(const Polar &P, const double dF[3][3], double out[3][3])
{
    double K[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) K[a][b] = P.R[0][a] * dF[0][b] + P.R[1][a] * dF[1][b] + P.R[2][a] * dF[2][b];
    const double a0 = K[2][1] - K[1][2], a1 = K[0][2] - K[2][0], a2 = K[1][0] - K[0][1];
    const double b0 = P.Mi[0][0] * a0 + P.Mi[0][1] * a1 + P.Mi[0][2] * a2;
    const double b1 = P.Mi[1][0] * a0 + P.Mi[1][1] * a1 + P.Mi[1][2] * a2;
    const double b2 = P.Mi[2][0] * a0 + P.Mi[2][1] * a1 + P.Mi[2][2] * a2;
    const double Bm[3][3] = {{0.0, -b2, b1}, {b2, 0.0, -b0}, {-b1, b0, 0.0}};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) out[a][b] = P.R[a][0] * Bm[0][b] + P.R[a][1] * Bm[1][b] + P.R[a][2] * Bm[2][b];
}

// the diagonal entry of vertex weight vector w and component c: a = w x rho, rho = R^T e_c (row c of R)
__device__ inline double polar_h1_diag(const Polar &P, const double w[3], int c)
{
    const double r0 = P.R[c][0], r1 = P.R[c][1], r2 = P.R[c][2];
    return quad_Mi(P, w[1] * r2 - w[2] * r1, w[2] * r0 - w[0] * r2, w[0] * r1 - w[1] * r0);
}

} // namespace pncg
