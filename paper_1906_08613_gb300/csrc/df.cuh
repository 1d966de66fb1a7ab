// Double-float arithmetic on the FP32 pipe.
//
// A double-float value is an unevaluated sum hi + lo of two floats, about 48
// significant bits.  FP64 operands are split into hi (the leading 24 bits of
// the significand) and lo (the next 24 bits), both by truncation and with
// integer operations only, so that splitting takes no FP64 instruction; the
// five dropped bits bound the representation error by 2^-47 relative.
// Products and sums use the error-free transformations TwoProduct (one FMA
// gives the exact rounding error of a product) and TwoSum (Knuth: six
// additions give the exact rounding error of a sum).
#pragma once

#include <cuda_runtime.h>

namespace ss {

// x -> (hi, lo).  Values outside the FP32 normal range (magnitude below about
// 1.2e-38 or above 3.4e38) take the hardware conversions instead and lose the
// double-float accuracy; lo flushes to zero when it would be subnormal.
__device__ __forceinline__ void split_df(double x, float &hi, float &lo)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(u >> 32) & 0x80000000u;
    const int e = (int)((u >> 52) & 0x7FF);
    const int ef = e - 896;                       // e - 1023 + 127
    if (ef >= 1 && ef <= 254) {
        hi = __uint_as_float(sgn | ((unsigned)ef << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
        const unsigned ml = (unsigned)(u & 0x1FFFFFFFu);
        if (ml == 0u) { lo = 0.0f; return; }
        const int lz = __clz(ml);                 // 3..31
        const int el = e - 1075 + (31 - lz) + 127;
        if (el >= 1) {
            const unsigned mant = (unsigned)((((unsigned long long)ml) << (lz + 1)) >> 9) & 0x7FFFFFu;
            lo = __uint_as_float(sgn | ((unsigned)el << 23) | mant);
        } else {
            lo = 0.0f;
        }
    } else if ((u << 1) == 0ull) {
        hi = 0.0f;
        lo = 0.0f;
    } else {
        hi = __double2float_rz(x);
        lo = __double2float_rn(x - (double)hi);
    }
}

// FP32 -> FP64 exactly, integer operations only (subnormal, infinite and NaN
// inputs take the hardware conversion).
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned v = __float_as_uint(f);
    const unsigned e = (v >> 23) & 0xFFu;
    if (e >= 1u && e <= 254u) {
        const unsigned long long u = ((unsigned long long)(v & 0x80000000u) << 32) |
                                     ((unsigned long long)(e + 896u) << 52) |
                                     ((unsigned long long)(v & 0x7FFFFFu) << 29);
        return __longlong_as_double((long long)u);
    }
    if ((v << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)(v & 0x80000000u) << 32));
    return (double)f;
}

// acc -= x * y in double-float (acc, x, y each hi + lo; the lo * lo term is
// below the format's precision and dropped).  The steps are never contracted
// into FMAs, so the error-free transformations stay exact.
__device__ __forceinline__ void df_msub(float &ah, float &al, float xh, float xl, float yh, float yl)
{
    const float p = __fmul_rn(xh, yh);
    float pe = __fmaf_rn(xh, yh, -p);                      // p + pe = xh * yh exactly
    pe = __fadd_rn(pe, __fmaf_rn(xh, yl, __fmul_rn(xl, yh)));
    const float s = __fsub_rn(ah, p);                      // TwoSum(ah, -p)
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    ah = s;
    al = __fadd_rn(al, __fsub_rn(err, pe));
}

// hi + lo rounded to FP64 (one FP64 addition).
__device__ __forceinline__ double df_to_double(float hi, float lo) { return f2d_exact(hi) + f2d_exact(lo); }

// a += b (TwoSum of the high parts, low parts added).
__device__ __forceinline__ void df_add(float &ah, float &al, float bh, float bl)
{
    const float s = __fadd_rn(ah, bh);
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    ah = s;
    al = __fadd_rn(al, __fadd_rn(bl, err));
}

// (h, l) -> the same sum with |l| <= ulp(h) / 2 (TwoSum of h and l).
__device__ __forceinline__ void df_norm(float &h, float &l)
{
    const float s = __fadd_rn(h, l);
    const float bb = __fsub_rn(s, h);
    l = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(l, bb));
    h = s;
}

// x = v * r for normalised v and r: TwoProduct of the high parts plus the two
// cross terms, then Fast2Sum (|p| >= |e|) to normalise.
__device__ __forceinline__ void df_mul(float vh, float vl, float rh, float rl, float &xh, float &xl)
{
    const float p = __fmul_rn(vh, rh);
    float e = __fmaf_rn(vh, rh, -p);
    e = __fmaf_rn(vh, rl, e);
    e = __fmaf_rn(vl, rh, e);
    const float s = __fadd_rn(p, e);
    xl = __fsub_rn(e, __fsub_rn(s, p));
    xh = s;
}

// Sum of (h, l) over the `split` consecutive lanes of a group (split a power
// of two dividing 32); every lane of the group gets the sum.
__device__ __forceinline__ void df_group_sum(float &h, float &l, int split)
{
    for (int o = split >> 1; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, h2, l2);
    }
}

}  // namespace ss
