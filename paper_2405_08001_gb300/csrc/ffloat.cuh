// Float-float ("double-float") helpers for the FP32 form: a value is carried as an unevaluated sum hi + lo of
// two floats.  Used to form vertex differences and the metric change Ds^T Ds - Dm^T Dm of a tet without FP64
// arithmetic.  The error-free transforms are Knuth's TwoSum / TwoDiff and the FMA-based TwoProd; the intrinsics
// (__fadd_rn, __fmul_rn, __fmaf_rn) keep the compiler from contracting or reassociating them.
#pragma once

namespace pncg {

struct ffl { float h, l; };

__device__ inline ffl ff_split(double d)
{
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}

// a - b exactly as an unevaluated sum (TwoDiff)
__device__ inline ffl two_diff(float a, float b)
{
    const float s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
    return {s, e};
}

// (ah + al) - (bh + bl) to about 2^-46 relative accuracy
__device__ inline ffl ff_sub(float ah, float al, float bh, float bl)
{
    ffl d = two_diff(ah, bh);
    d.l = __fadd_rn(d.l, __fsub_rn(al, bl));
    const float s = __fadd_rn(d.h, d.l);
    return {s, __fsub_rn(d.l, __fsub_rn(s, d.h))};
}

__device__ inline float ff_val(ffl a) { return __fadd_rn(a.h, a.l); }

// (h + l) += (ah + al) p: the head product exact (FMA TwoProd), its tail and al p joined to the error of the TwoSum
// of the heads, then renormalised (about 2^-46 relative accuracy)
__device__ inline void ff_axpy(float &h, float &l, float ah, float al, float p)
{
    const float q = __fmul_rn(ah, p);
    float e = __fmaf_rn(al, p, __fmaf_rn(ah, p, -q));
    const float s = __fadd_rn(h, q), bb = __fsub_rn(s, h);
    e = __fadd_rn(e, __fadd_rn(__fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(q, bb)), l));
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

// Compensated accumulator: s + c carries sum_k sign_k x_k y_k for float-float x, y.  The first term can start it
// (prod, prod_f): the TwoSum of a term into a zero sum is exact and only costs instructions.
struct ffacc {
    float s = 0.0f, c = 0.0f;
    // x y for float-float x, y: the FMA TwoProd of the heads, the cross terms into the compensation
    __device__ static inline ffacc prod(ffl x, ffl y)
    {
        ffacc a;
        a.s = __fmul_rn(x.h, y.h);
        float e = __fmaf_rn(x.h, y.h, -a.s);
        e = __fmaf_rn(x.h, y.l, e);
        a.c = __fmaf_rn(x.l, y.h, e);
        return a;
    }
    // x y for a float-float x and a float y
    __device__ static inline ffacc prod_f(ffl x, float y)
    {
        ffacc a;
        a.s = __fmul_rn(x.h, y);
        a.c = __fmaf_rn(x.l, y, __fmaf_rn(x.h, y, -a.s));
        return a;
    }
    __device__ inline void add_prod(ffl x, ffl y, float sign)
    {
        float p = __fmul_rn(x.h, y.h);
        float e = __fmaf_rn(x.h, y.h, -p);
        e = __fmaf_rn(x.h, y.l, e);
        e = __fmaf_rn(x.l, y.h, e);
        p = __fmul_rn(p, sign);
        e = __fmul_rn(e, sign);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    // adds x y for a float-float x and a float y (Dot2: the FMA TwoProd of the heads, the tail's product into the
    // compensation)
    __device__ inline void add_prod_f(ffl x, float y)
    {
        const float p = __fmul_rn(x.h, y);
        float e = __fmaf_rn(x.h, y, -p);
        e = __fmaf_rn(x.l, y, e);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ inline ffl ff() const { return {s, c}; }
    // subtracts the float-float value h + l
    __device__ inline void sub_ff(float h, float l)
    {
        const float p = -h;
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fsub_rn(err, l));
    }
    __device__ inline float value() const { return __fadd_rn(s, c); }
};

// A float-float number with arithmetic, for re-evaluating the closest-point geometry of active contact pairs in the
// FP32 form (Sec. 3.2 templates instantiated on it): about 2^-44 relative accuracy on the FP32 pipes.  Addition
// is TwoSum of the heads plus the tails, multiplication the FMA TwoProd plus cross terms, division and square root
// one correction step of the float quotient / root (Dekker's double-length arithmetic).
struct ffn {
    float h, l;
    __host__ __device__ ffn() : h(0.0f), l(0.0f) {}
    __host__ __device__ explicit ffn(float a) : h(a), l(0.0f) {}
    __host__ __device__ explicit ffn(double a) : h((float)a), l((float)(a - (double)(float)a)) {}
    __host__ __device__ explicit ffn(int a) : h((float)a), l(0.0f) {}
    __device__ ffn(float a, float b) : h(a), l(b) {}
};

__device__ inline ffn ffn_renorm(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return ffn(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ inline ffn operator+(ffn a, ffn b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return ffn_renorm(s, e);
}
__device__ inline ffn operator-(ffn a) { return ffn(-a.h, -a.l); }
__device__ inline ffn operator-(ffn a, ffn b) { return a + (-b); }
__device__ inline ffn operator*(ffn a, ffn b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ffn_renorm(p, e);
}
__device__ inline ffn operator/(ffn a, ffn b)
{
    const float q1 = __fdiv_rn(a.h, b.h);
    const ffn r = a - b * ffn(q1);
    const float q2 = __fdiv_rn(r.h, b.h);
    return ffn_renorm(q1, q2);
}
__device__ inline ffn gsqrt(ffn a)
{
    if (!(a.h > 0.0f)) return ffn(0.0f);
    const float s = __fsqrt_rn(a.h);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);
    const ffn r = a - ffn(p, pe);
    return ffn_renorm(s, __fdiv_rn(r.h, __fmul_rn(2.0f, s)));
}
__device__ inline bool operator<(ffn a, ffn b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ inline bool operator>(ffn a, ffn b) { return b < a; }
__device__ inline bool operator<=(ffn a, ffn b) { return !(b < a); }
__device__ inline bool operator>=(ffn a, ffn b) { return !(a < b); }

} // namespace pncg
