// Double-word ("float-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi)/2, which carries about 48 significant bits.  The building blocks
// are the error-free transformations of the literature: TwoSum (Knuth, TAOCP vol. 2,
// Sec. 4.2.2), Fast2Sum (Dekker 1971, for |a| >= |b|) and the exact product
// a*b = p + e with e = fma(a, b, -p).  Each double-word operation below is one of the
// standard combinations of these (e.g. Joldes, Muller & Popescu, ACM TOMS 44 (2017):
// the "sloppy" sum, whose error is bounded relative to |x| + |y| rather than to the
// result, and the product with one cross term dropped).
//
// On GB300 the FP32 pipe executes 64 times as many lanes per cycle as the FP64 pipe,
// so a double-word operation of 6-15 FP32 instructions costs a fraction of one FP64
// instruction's issue time.  The implicit solve uses it to form a Newton correction
// from a residual accurate to ~1e-14; the root itself is still accepted only by the
// FP64 residual.
//
// Every sum and product goes through the __f*_rn intrinsics or fmaf so that the
// compiler neither contracts nor reorders them (the transformations rely on each
// operation being rounded exactly once, as written).
#pragma once

namespace grmhd {

struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw dw_make(float a) { return {a, 0.0f}; }

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ dw two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// a + b = s + e exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ dw fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dw dw_add(dw x, dw y)
{
    const dw s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ dw dw_neg(dw x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }

__device__ __forceinline__ dw dw_add_f(dw x, float b)
{
    const dw s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ dw dw_mul(dw x, dw y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dw dw_mul_f(dw x, float b)
{
    const float p = __fmul_rn(x.hi, b);
    float e = fmaf(x.hi, b, -p);
    e = fmaf(x.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dw dw_sqr(dw x)
{
    const float p = __fmul_rn(x.hi, x.hi);
    float e = fmaf(x.hi, x.hi, -p);
    e = fmaf(__fadd_rn(x.hi, x.hi), x.lo, e);
    return fast_two_sum(p, e);
}

// x * 2^k for a power-of-two factor s (exact unless it leaves the normal range)
__device__ __forceinline__ dw dw_scale(dw x, float s) { return {__fmul_rn(x.hi, s), __fmul_rn(x.lo, s)}; }

// 1/x: y0 = 1/x.hi to ~1 ulp, then one Newton correction y0 + y0 (1 - x y0) with the
// residual 1 - x y0 formed by fused multiply-adds (quadratic: ~2^-46 relative)
__device__ __forceinline__ dw dw_rcp(dw x)
{
    const float y = __frcp_rn(x.hi);
    float r = fmaf(-x.hi, y, 1.0f);
    r = fmaf(-x.lo, y, r);
    return fast_two_sum(y, __fmul_rn(y, r));
}

// sqrt(x) for x > 0: h = sqrt(x.hi) correctly rounded, then h + (x - h^2)/(2h) with
// x - h^2 formed exactly from the product error
__device__ __forceinline__ dw dw_sqrt(dw x)
{
    const float h = __fsqrt_rn(x.hi);
    const float p = __fmul_rn(h, h);
    const float e = fmaf(h, h, -p);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), e), x.lo);
    // the correction is ~2^-24 h, so an approximate 0.5/h suffices
    return fast_two_sum(h, __fmul_rn(d, __fdividef(0.5f, h)));
}

}  // namespace grmhd
