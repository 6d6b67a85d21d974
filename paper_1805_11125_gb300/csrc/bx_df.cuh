// bx_df.cuh -- double-float arithmetic in FP32 (value h + l, |l| <= ulp(h) / 2): ~2^-44 relative
// precision at FP32 issue cost, for the per-column quantities that need more than FP32 but not
// FP64 (GB300 issues FP64 at 1/64 of its FP32 rate).  Error-free transformations:
// TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|), TwoProduct by FMA; reciprocal and
// reciprocal square root by one Newton step from the FP32 value.
#pragma once

#ifdef __CUDACC__

namespace bx {

struct df {
    float h, l;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_fast(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = df_two_sum(a.h, b.h);
    return df_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df df_addf(df a, float b) {
    const df s = df_two_sum(a.h, b);
    return df_fast(s.h, __fadd_rn(s.l, a.l));
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return df_fast(p, e);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = __fmul_rn(a.h, b);
    return df_fast(p, fmaf(a.l, b, fmaf(a.h, b, -p)));
}
// 1 / a: r0 = 1/a.h in FP32, then r = r0 + r0 (1 - a r0) in double-float
__device__ __forceinline__ df df_recip(df a) {
    const float r0 = __frcp_rn(a.h);
    const df e = df_addf(df_neg(df_mulf(a, r0)), 1.0f);
    return df_addf(df_mulf(e, r0), r0);
}
// 1 / sqrt(a): r0 from FP32, then r = r0 + r0 (1 - a r0^2) / 2 in double-float
__device__ __forceinline__ df df_rsqrt(df a) {
    float r0 = rsqrtf(a.h);
    r0 = fmaf(0.5f * r0, fmaf(-a.h * r0, r0, 1.0f), r0);   // FP32 step: r0 to ~1 ulp
    const df e = df_addf(df_neg(df_mulf(df_mulf(a, r0), r0)), 1.0f);
    return df_addf(df_mulf(e, 0.5f * r0), r0);
}
__device__ __forceinline__ df df_from(double x) {
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}
// Exact float -> double through the bit fields (integer pipe; the conversion instruction
// shares GB300's FP64 pipe): zero and normal floats; subnormal, infinite and NaN inputs take
// the conversion instruction.
__device__ __forceinline__ double f2d(float x) {
    const unsigned u = __float_as_uint(x), e = (u >> 23) & 0xffu;
    if (e - 1u >= 0xfeu) {   // e == 0 or e == 255
        if ((u << 1) == 0u) return __hiloint2double((int)u, 0);
        return (double)x;
    }
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}
__device__ __forceinline__ double df_to_double(df a) { return f2d(a.h) + f2d(a.l); }

}  // namespace bx

#endif  // __CUDACC__
