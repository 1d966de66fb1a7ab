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

// x * 2^sh -> (hi, lo), the power-of-two scaling folded into the exponent
// (one integer addition more than split_df).  This is how the double-float
// pipelines read every FP64 operand: each instance is rescaled by powers of
// two so that its largest entries lie in [1, 2) (see DfScale), which keeps
// operands, products and sums inside FP32's exponent range whatever the
// magnitude of the FP64 data.  A scaled value below 2^-126 (or an FP64
// subnormal) becomes 0: an absolute error under 2^-126 against entries of
// order one.  A scaled value of 2^128 or more becomes +-Inf, and Inf or NaN
// stays Inf or NaN (lo = 0), so that the caller's range check sees it.
__device__ __forceinline__ void split_df_s(double x, int sh, float &hi, float &lo)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(u >> 32) & 0x80000000u;
    const int e = (int)((u >> 52) & 0x7FF);
    const int ef = e - 896 + sh;                  // e - 1023 + 127 + sh
    if (e != 0 && e != 0x7FF && ef >= 1 && ef <= 254) {
        hi = __uint_as_float(sgn | ((unsigned)ef << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
        const unsigned ml = (unsigned)(u & 0x1FFFFFFFu);
        lo = 0.0f;
        if (ml != 0u) {
            const int lz = __clz(ml);             // 3..31
            const int el = ef - 52 + (31 - lz);   // exponent of the leading bit of ml
            if (el >= 1) {
                const unsigned mant = (unsigned)((((unsigned long long)ml) << (lz + 1)) >> 9) & 0x7FFFFFu;
                lo = __uint_as_float(sgn | ((unsigned)el << 23) | mant);
            }
        }
    } else if (e == 0x7FF) {
        hi = __double2float_rn(x);
        lo = 0.0f;
    } else if (e != 0 && ef > 254) {
        hi = __uint_as_float(sgn | 0x7F800000u);
        lo = 0.0f;
    } else {
        hi = __uint_as_float(sgn);
        lo = 0.0f;
    }
}

// Biased FP64 exponent of x (0 for zero and subnormals, 0x7FF for Inf / NaN).
__device__ __forceinline__ int exp_bits(double x)
{
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
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

// f * 2^sh in FP64, exact whenever the result is an FP64 normal number
// (integer operations; other cases take ldexp).
__device__ __forceinline__ double f2d_exact_s(float f, int sh)
{
    const unsigned v = __float_as_uint(f);
    const int e = (int)((v >> 23) & 0xFFu);
    const int ed = e + 896 + sh;
    if (e >= 1 && e <= 254 && ed >= 1 && ed <= 2046) {
        const unsigned long long u = ((unsigned long long)(v & 0x80000000u) << 32) |
                                     ((unsigned long long)ed << 52) |
                                     ((unsigned long long)(v & 0x7FFFFFu) << 29);
        return __longlong_as_double((long long)u);
    }
    if ((v << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)(v & 0x80000000u) << 32));
    return ldexp((double)f, sh);
}

// (hi + lo) * 2^sh rounded to FP64: the scaled value of a double-float
// result back in the caller's units.
__device__ __forceinline__ double df_to_double_s(float hi, float lo, int sh)
{
    return f2d_exact_s(hi, sh) + f2d_exact_s(lo, sh);
}

// True if |v| >= 2^60 or v is Inf / NaN: a double-float intermediate of a
// rescaled instance has left the range in which products with operands of
// order one keep their absolute error below 2^-66 (see DfScale).
__device__ __forceinline__ bool df_out_of_range(float v)
{
    return (__float_as_uint(v) & 0x7F800000u) >= ((127u + 60u) << 23);
}

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
