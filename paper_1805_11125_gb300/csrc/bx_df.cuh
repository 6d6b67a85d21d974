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
// a / b: q0 = a.h / b.h, then one correction from the double-float residual a - q0 b
__device__ __forceinline__ df df_div(df a, df b) {
    const float q0 = __fdiv_rn(a.h, b.h);
    const df r = df_add(a, df_neg(df_mulf(b, q0)));
    return df_fast(q0, __fdiv_rn(r.h, b.h));
}
// ln r for r > 0 with 1e-30 <= r.h <= 1e30, ~2e-11 relative: r = 2^e m with m in
// [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s) with s = (m - 1)/(m + 1), |s| <= 0.1716:
// 2s + (2/3) s^3 in double-float, the rest s^5 (2/5 + 2 s^2/7 + ... + 2 s^12/17) in FP32
// (at most 2e-4 of ln m; truncation below 1e-13 of it); e ln 2 with ln 2 as a double-float.
__device__ __forceinline__ df df_log(df r) {
    const unsigned u = __float_as_uint(r.h);
    int e = (int)((u >> 23) & 0xffu) - 127;
    unsigned mb = (u & 0x007fffffu) | 0x3f800000u;
    if (__uint_as_float(mb) > 1.41421356f) {
        mb -= 0x00800000u;
        e += 1;
    }
    const df m{__uint_as_float(mb), r.l * __uint_as_float((unsigned)(127 - e) << 23)};
    const df s = df_div(df_addf(m, -1.0f), df_addf(m, 1.0f));
    const df s2 = df_mul(s, s), s3 = df_mul(s2, s);
    float q = 2.0f / 17.0f;
    q = fmaf(s2.h, q, 2.0f / 15.0f);
    q = fmaf(s2.h, q, 2.0f / 13.0f);
    q = fmaf(s2.h, q, 2.0f / 11.0f);
    q = fmaf(s2.h, q, 2.0f / 9.0f);
    q = fmaf(s2.h, q, 2.0f / 7.0f);
    q = fmaf(s2.h, q, 2.0f / 5.0f);
    const df two3{0.6666666865348816f, -1.9868215517249155e-08f};
    const df lm = df_addf(df_add(df{2.0f * s.h, 2.0f * s.l}, df_mul(s3, two3)), s3.h * s2.h * q);
    const df ln2{0.6931471824645996f, -1.9046542121259336e-09f};
    return df_add(df_mulf(ln2, (float)e), lm);
}

// Baker-Cousins term mu - n + n ln(n/mu) (n > 0, mu > 0) and w = 1 - n/mu in double-float,
// ~1e-11 relative (the two parts are within a factor ~5 of the term wherever n/mu lies
// outside [1/2, 2]).  Returns false where n/mu is beyond [1e-30, 1e30].
__device__ __forceinline__ bool bc_term_far(df n, df mu, df& term, float& wb) {
    const df r = df_div(n, mu);
    if (!(r.h >= 1e-30f && r.h <= 1e30f)) return false;
    term = df_add(df_add(mu, df_neg(n)), df_mul(n, df_log(r)));
    wb = 1.0f - r.h;
    return true;
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
