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

// Compensated accumulator: s + c carries sum_k sign_k x_k y_k for float-float x, y.
struct ffacc {
    float s = 0.0f, c = 0.0f;
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
    __device__ inline float value() const { return __fadd_rn(s, c); }
};

} // namespace pncg
