// Contact geometry of Sec. 3.2: the unified point-triangle / edge-edge distance d = |t|, t = sum c_i x_i, and the
// IPC log barrier (Eq. barrier) with its first two derivatives.  Host + device templates (R = float, double, or
// the float-float number type of the FP32 form).
#pragma once

#include <math.h>

namespace pncg {

template <typename R> struct v3 { R x, y, z; };

// square root of the geometry's number type (float, double, or the float-float type of the FP32 form)
__host__ __device__ inline float gsqrt(float a) { return sqrtf(a); }
__host__ __device__ inline double gsqrt(double a) { return ::sqrt(a); }

template <typename R> __host__ __device__ inline v3<R> mkv(R a, R b, R c) { v3<R> r; r.x = a; r.y = b; r.z = c; return r; }

// Relative size of the 2x2 normal equations' determinant below which the interior solution is not trusted (nearly
// parallel edges, a sliver triangle) and the clamped cases decide.  It must exceed the determinant's rounding error,
// a few units of the number type's precision relative to a cq: 1e-12 for double and the float-float type (2^-44),
// 1e-5 for float (2^-24), whose interior solution of two parallel edges can otherwise come out of cancellation noise.
template <typename R> struct GeomEps { static constexpr double par = 1e-12; };
template <> struct GeomEps<float> { static constexpr double par = 1e-5; };
template <typename R> __host__ __device__ inline v3<R> operator-(v3<R> a, v3<R> b) { return mkv(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename R> __host__ __device__ inline v3<R> operator+(v3<R> a, v3<R> b) { return mkv(a.x + b.x, a.y + b.y, a.z + b.z); }
template <typename R> __host__ __device__ inline v3<R> operator*(R s, v3<R> a) { return mkv(s * a.x, s * a.y, s * a.z); }
template <typename R> __host__ __device__ inline R dot(v3<R> a, v3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename R> __host__ __device__ inline v3<R> cross(v3<R> a, v3<R> b)
{
    return mkv(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Closest point of segment [a, b] to q: returns the squared distance and the parameter u in [0, 1].
template <typename R> __host__ __device__ inline R seg_closest(v3<R> q, v3<R> a, v3<R> b, R &u)
{
    v3<R> ab = b - a, aq = q - a;
    R L2 = dot(ab, ab);
    R s = L2 > R(0) ? dot(aq, ab) / L2 : R(0);
    s = s < R(0) ? R(0) : (s > R(1) ? R(1) : s);
    v3<R> r = aq - s * ab;
    u = s;
    return dot(r, r);
}

// Point-triangle in coordinates relative to the triangle's first vertex:
//   r = x0 - x1 (the point), e1 = x2 - x1, e2 = x3 - x1.
// Minimises |x0 - (a x1 + b x2 + g x3)| over the simplex (Eq. PT); c = (1, -a, -b, -g).  Interior projection from
// the 2x2 normal equations when it lies in the triangle, else the closest of the three clamped edges in the
// order (x1,x2), (x2,x3), (x3,x1) (first wins ties).  Returns d and writes c and t = x0 - x_b.
template <typename R> __host__ __device__ inline R pt_coeffs(v3<R> r, v3<R> e1, v3<R> e2, R c[4], v3<R> &t)
{
    R a = dot(e1, e1), b = dot(e1, e2), cq = dot(e2, e2);
    R det = a * cq - b * b;
    if (det > R(GeomEps<R>::par) * a * cq) {
        R p = dot(r, e1), q = dot(r, e2);
        R be = (cq * p - b * q) / det, ga = (a * q - b * p) / det;
        if (be >= R(0) && ga >= R(0) && be + ga <= R(1)) {
            c[0] = R(1); c[1] = -(R(1) - be - ga); c[2] = -be; c[3] = -ga;
            t = r - (be * e1 + ga * e2);
            return gsqrt(dot(t, t));
        }
    }
    v3<R> zero = mkv(R(0), R(0), R(0));
    R u, best;
    // edge x1-x2
    best = seg_closest(r, zero, e1, u);
    c[0] = R(1); c[1] = -(R(1) - u); c[2] = -u; c[3] = R(0);
    // edge x2-x3
    R d2 = seg_closest(r, e1, e2, u);
    if (d2 < best) { best = d2; c[1] = R(0); c[2] = -(R(1) - u); c[3] = -u; }
    // edge x3-x1
    d2 = seg_closest(r, e2, zero, u);
    if (d2 < best) { best = d2; c[1] = -u; c[2] = R(0); c[3] = -(R(1) - u); }
    t = r + c[2] * e1 + c[3] * e2;
    return gsqrt(dot(t, t));
}

// Edge-edge in coordinates relative to x2 (first vertex of the second edge):
//   r = x0 - x2, a1 = x1 - x2, e1 = x3 - x2.
// Minimises |(1-s) x0 + s x1 - ((1-u) x2 + u x3)| over [0,1]^2 (Eq. EE); c = (1-s, s, -(1-u), -u).  Interior
// solution of the 2x2 system when it lies in the square (and the edges are not parallel), else the closest of the
// four clamped cases s = 0, s = 1, u = 0, u = 1 in that order.  Returns d and writes c and t.
template <typename R> __host__ __device__ inline R ee_coeffs(v3<R> r, v3<R> a1, v3<R> e1, R c[4], v3<R> &t)
{
    v3<R> e0 = a1 - r;
    R a = dot(e0, e0), b = dot(e0, e1), cq = dot(e1, e1), dd = dot(e0, r), ee = dot(e1, r);
    R det = a * cq - b * b;
    bool done = false;
    if (det > R(GeomEps<R>::par) * a * cq) {
        R s = (b * ee - cq * dd) / det, u = (a * ee - b * dd) / det;
        if (s >= R(0) && s <= R(1) && u >= R(0) && u <= R(1)) {
            c[0] = R(1) - s; c[1] = s; c[2] = -(R(1) - u); c[3] = -u;
            done = true;
        }
    }
    if (!done) {
        v3<R> zero = mkv(R(0), R(0), R(0));
        R u, best, d2;
        best = seg_closest(r, zero, e1, u);          // s = 0: x0 against x2-x3
        c[0] = R(1); c[1] = R(0); c[2] = -(R(1) - u); c[3] = -u;
        d2 = seg_closest(a1, zero, e1, u);           // s = 1: x1 against x2-x3
        if (d2 < best) { best = d2; c[0] = R(0); c[1] = R(1); c[2] = -(R(1) - u); c[3] = -u; }
        d2 = seg_closest(zero, r, a1, u);            // u = 0: x2 against x0-x1
        if (d2 < best) { best = d2; c[0] = R(1) - u; c[1] = u; c[2] = R(-1); c[3] = R(0); }
        d2 = seg_closest(e1, r, a1, u);              // u = 1: x3 against x0-x1
        if (d2 < best) { best = d2; c[0] = R(1) - u; c[1] = u; c[2] = R(0); c[3] = R(-1); }
    }
    t = c[0] * r + c[1] * a1 + c[3] * e1;
    return gsqrt(dot(t, t));
}

// Relative coordinates of a pair from double positions, rounded to R after the subtraction.
template <typename R> __host__ __device__ inline v3<R> rel(double ax, double ay, double az, double bx, double by, double bz)
{
    return mkv(R(ax - bx), R(ay - by), R(az - bz));
}

// b(d) = -(d - dhat)^2 log(d/dhat) for 0 < d < dhat: first and second derivative in d, from d and r = d - dhat.
// log(d/dhat) is formed as log1p(r/dhat), which keeps its relative accuracy as d -> dhat when r is accurate (the
// FP32 form passes r from its float-float distance: a float d has lost r's low bits near the cut-off).
template <typename R> __host__ __device__ inline void barrier_d12r(R d, R r, R dhat, R &b1, R &b2)
{
    const R L = log1p(r / dhat);
    b1 = R(-2) * r * L - r * r / d;
    b2 = R(-2) * L - R(4) * r / d + (r * r) / (d * d);
}
template <typename R> __host__ __device__ inline void barrier_d12(R d, R dhat, R &b1, R &b2)
{
    barrier_d12r<R>(d, d - dhat, dhat, b1, b2);
}

template <typename R> __host__ __device__ inline R barrier_b(R d, R dhat)
{
    R r = d - dhat;
    return -r * r * log1p(r / dhat);
}

} // namespace pncg
