// bx_resp.cuh -- FP32 generation of the response entries (Eq. 1) without hardware
// approximations: every operation is a round-to-nearest FMA/add/multiply, so the
// rounding errors carry no systematic sign.
//
// Bin mass of the Gaussian of column i over output bin m, by 3-point Gauss-Legendre
// quadrature of its density (nodes c, c -+ (h/2) sqrt(3/5), weights 8/9, 5/9, 5/9),
// in the scaled variable t = z * S_EX2 so that exp(-z^2/2) = 2^(-t^2):
//   p0  = 2^(-t0^2)                               centre node
//   p-+ = p0 * 2^(-kk^2) * 2^(+-2 kk t0)          outer nodes, kk = sqrt(3/5)/2 * hs
//   p- + p+ = p0 * Ck2 * cosh(z),  Ck2 = 2 * 2^(-kk^2),  z = 2 ln2 kk t0 = kap t0
//   p- - p+ = p0 * Ck2 * sinh(z)
//   R   = A * (8 p0 + 5 (p- + p+)),  A = (h/2) norm / (9 sqrt(2 pi))   (weights as exact integers)
// The centre-node exponent t0^2 is formed in double-float (error-free transformations by FMA)
// from double-float column parameters: in plain FP32 its rounding alone gives a relative
// error q ln2 2^-24 in 2^(-q), ~3e-7 per entry.
// 2^x (x <= 0) uses Cody-Waite reduction x = n + f, |f| <= 1/2, a degree-7 polynomial for
// 2^f (coefficients fitted by weighted least squares on [-1/2, 1/2], approximation error
// 4e-11) and the exponent field for 2^n.  cosh and sinh use their Taylor series through
// z^10 / z^11 (truncation < 2e-9 for |z| <= 1); larger |z| (only for very narrow
// resolutions) evaluates the two outer nodes directly with the same exp2.
#pragma once

#include "bx_internal.cuh"

namespace bx {

#ifdef __CUDACC__

// 2^(xh + xl) for xh <= 0 (double-float argument, |xl| << 1).
__device__ __forceinline__ float exp2_neg(float xh, float xl = 0.0f) {
    xh = fmaxf(xh, -127.0f);
    const float t = __fadd_rn(xh, 12582912.0f);   // 1.5 * 2^23: n = rint(xh) lands in the low bits
    const float n = __fsub_rn(t, 12582912.0f);
    const float f = __fadd_rn(__fsub_rn(xh, n), xl);   // |f| <= 1/2 + |xl|
    float p = 1.520192109e-05f;
    p = fmaf(p, f, 1.546929125e-04f);
    p = fmaf(p, f, 1.333392225e-03f);
    p = fmaf(p, f, 9.618027136e-03f);
    p = fmaf(p, f, 5.550410226e-02f);
    p = fmaf(p, f, 2.402265072e-01f);
    p = fmaf(p, f, 6.931471825e-01f);
    p = fmaf(p, f, 1.0f);
    // 2^n from the exponent field: bits(t) = 0x4B400000 + n; n = -127 gives +0
    const int e = (__float_as_int(t) - 0x4B400000 + 127) << 23;
    return __fmul_rn(p, __int_as_float(e));
}

// Scaled centre-node position t0 = (m + 1/2 - mu/w) * hs of output bin m as a double-float
// (th, tl): k = m - floor(mu/w) is an exact integer, hs = hs_hi + hs_lo and
// c = (1/2 - frac(mu/w)) hs = c_hi + c_lo come from FP64; products and sums are error-free
// transformations (TwoProduct by FMA, TwoSum), so th + tl carries ~2^-40 relative error.
__device__ __forceinline__ void centre_df(float mf, const float4& cf, float c_lo, float& th, float& tl) {
    const float k = __fsub_rn(mf, cf.x);
    const float p = __fmul_rn(k, cf.z);
    float e = fmaf(k, cf.z, -p);
    e = fmaf(k, cf.w, e);
    const float s = __fadd_rn(p, cf.y);
    const float bb = __fsub_rn(s, p);
    const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(cf.y, bb));
    th = s;
    tl = __fadd_rn(__fadd_rn(err, e), c_lo);
}

// p0 = 2^(-t0^2) with the square and the reduction carried in double-float.
__device__ __forceinline__ float centre_node(float th, float tl) {
    const float qh = __fmul_rn(th, th);
    const float qe = fmaf(th, th, -qh);
    const float ql = fmaf(__fadd_rn(th, th), tl, qe);
    return exp2_neg(-qh, -ql);
}

__device__ __forceinline__ float cosh_small(float s) {   // s = z^2
    float c = 2.755731922e-07f;                          // 1/10!
    c = fmaf(c, s, 2.480158730e-05f);                    // 1/8!
    c = fmaf(c, s, 1.388888889e-03f);                    // 1/6!
    c = fmaf(c, s, 4.166666667e-02f);                    // 1/4!
    c = fmaf(c, s, 0.5f);
    return fmaf(c, s, 1.0f);
}

__device__ __forceinline__ float sinh_small(float z, float s) {
    float c = 2.505210839e-08f;                          // 1/11!
    c = fmaf(c, s, 2.755731922e-06f);                    // 1/9!
    c = fmaf(c, s, 1.984126984e-04f);                    // 1/7!
    c = fmaf(c, s, 8.333333333e-03f);                    // 1/5!
    c = fmaf(c, s, 1.666666667e-01f);                    // 1/3!
    return z * fmaf(c, s, 1.0f);
}

// Outer-node sum S+ = p- + p+ and difference S- = p- - p+ (p-+ = 2^(-(t0 -+ kk)^2)).
// Small |z|: from p0 and the series; otherwise (very narrow resolution only) directly.
static __device__ __noinline__ void outer_direct(float t0, float kk, float& Sp, float& Sm) {
    const float a = t0 - kk, b = t0 + kk;
    const float pm = exp2_neg(-(a * a)), pp = exp2_neg(-(b * b));
    Sp = pm + pp;
    Sm = pm - pp;
}

constexpr float INV_2LN2 = 0.72134752044448170f;   // kk = kap / (2 ln 2)

// Response entry of output bin `mf` (row index as float) and one column, divided by the
// column's amplitude A: the node sum 8 p0 + 5 (p- + p+).
// cf = (floor(mu/w), c_hi, hs_hi, hs_lo); cg = (kap, Ck2, c_lo, A / 9).
// WIDE: the caller has established |z| <= 1 for this row (the series branch), so the test
// is skipped; the arithmetic is the same either way.
template <bool WIDE = false>
__device__ __forceinline__ float resp_shape32_t(float th, float tl, const ColG& cg) {
    const float p0 = centre_node(th, tl);
    const float z = cg.kap * th;
    float Sp;
    if (WIDE || fabsf(z) <= 1.0f) {
        Sp = p0 * cg.Ck2 * cosh_small(z * z);
    } else {
        float Sm;
        outer_direct(th, cg.kap * INV_2LN2, Sp, Sm);
    }
    return fmaf(GL_W_OUT, Sp, GL_W_MID * p0);
}
template <bool WIDE = false>
__device__ __forceinline__ float resp_shape32(float mf, const float4& cf, const ColG& cg) {
    float th, tl;
    centre_df(mf, cf, cg.c_lo, th, tl);
    return resp_shape32_t<WIDE>(th, tl, cg);
}
// The centre of row m + 32 from that of row m: t + 32 hs as a double-float (32 hs is exact).
__device__ __forceinline__ void centre_step32(float th, float tl, const float4& cf, float& uh, float& ul) {
    const float d = 32.0f * cf.z;
    const float s = __fadd_rn(th, d);
    const float bb = __fsub_rn(s, th);
    const float err = __fadd_rn(__fsub_rn(th, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    uh = s;
    ul = __fadd_rn(err, fmaf(32.0f, cf.w, tl));
}
// Response entry R[m, i] of output bin `mf` and one column.
// Gram-Charlier response (density phi(z) g(z), g = 1 + c3 He3(z) + c4 He4(z), c3 = skewness / 6,
// c4 = excess kurtosis / 24): the same three nodes, each density times g at its standard score
// z = t / S_EX2.  With Sp = p- + p+ and Sm = p- - p+ (p- at t0 - kk, p+ at t0 + kk):
//   p- g- + p+ g+ = Sp (g- + g+) / 2 + Sm (g- - g+) / 2.
__device__ __forceinline__ float gc_factor(float z, float c3, float c4) {
    const float z2 = z * z;
    return fmaf(c3, z * (z2 - 3.0f), fmaf(c4, fmaf(z2, z2 - 6.0f, 3.0f), 1.0f));
}
__device__ __forceinline__ float gc_slope(float z, float c3, float c4) {   // dg/dz = 3 c3 He2 + 4 c4 He3
    const float z2 = z * z;
    return fmaf(3.0f * c3, z2 - 1.0f, 4.0f * c4 * z * (z2 - 3.0f));
}
constexpr float INV_S_EX2 = 1.17741002251547469101f;   // 1 / S_EX2 = sqrt(2 ln 2)

template <bool WIDE = false>
__device__ __forceinline__ float resp_shape32_gc_t(float th, float tl, const ColG& cg, float c3, float c4) {
    const float p0 = centre_node(th, tl);
    const float z = cg.kap * th, kk = cg.kap * INV_2LN2;
    float Sp, Sm;
    if (WIDE || fabsf(z) <= 1.0f) {
        const float q = z * z, f = p0 * cg.Ck2;
        Sp = f * cosh_small(q);
        Sm = f * sinh_small(z, q);
    } else {
        outer_direct(th, kk, Sp, Sm);
    }
    const float z0 = th * INV_S_EX2, d = kk * INV_S_EX2;
    const float gm = gc_factor(z0 - d, c3, c4), gp = gc_factor(z0 + d, c3, c4);
    const float outer = fmaf(Sp, gm + gp, Sm * (gm - gp)) * 0.5f;
    return fmaf(GL_W_OUT, outer, GL_W_MID * p0 * gc_factor(z0, c3, c4));
}
template <bool WIDE = false>
__device__ __forceinline__ float resp_shape32_gc(float mf, const float4& cf, const ColG& cg, float c3, float c4) {
    float th, tl;
    centre_df(mf, cf, cg.c_lo, th, tl);
    return resp_shape32_gc_t<WIDE>(th, tl, cg, c3, c4);
}

// The adjoint node sums of the Gram-Charlier response for one row: with the standard score z of
// each node, P0 = sum w p g, P1 = S_EX2 sum w p (z g - g'), P2 = S_EX2^2 sum w p (z^2 g - z g')
// (g = 1 gives resp_adjoint32's sums), so that the chain rule of the Gaussian adjoint applies
// unchanged: d(p g)/dmu ~ p (z g - g'), d(p g / sigma)/dsigma ~ p ((z^2 - 1) g - z g').
__device__ __forceinline__ void resp_adjoint32_gc(float mf, const float4& cf, const ColG& cg, float c3, float c4,
                                                  float& P0, float& P1, float& P2) {
    float th, tl;
    centre_df(mf, cf, cg.c_lo, th, tl);
    const float p0 = centre_node(th, tl);
    const float z = cg.kap * th, kk = cg.kap * INV_2LN2;
    float Sp, Sm;
    if (fabsf(z) <= 1.0f) {
        const float q = z * z, f = p0 * cg.Ck2;
        Sp = f * cosh_small(q);
        Sm = f * sinh_small(z, q);
    } else {
        outer_direct(th, kk, Sp, Sm);
    }
    const float pm = 0.5f * (Sp + Sm), pp = 0.5f * (Sp - Sm);
    const float z0 = th * INV_S_EX2, d = kk * INV_S_EX2, zm = z0 - d, zp = z0 + d;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    auto node = [&](float w, float p, float zz) {
        const float g = gc_factor(zz, c3, c4), gs = gc_slope(zz, c3, c4);
        const float a = fmaf(zz, g, -gs);    // z g - g'
        s0 = fmaf(w * p, g, s0);
        s1 = fmaf(w * p, a, s1);
        s2 = fmaf(w * p, zz * a, s2);        // z^2 g - z g'
    };
    node(GL_W_MID, p0, z0);
    node(GL_W_OUT, pm, zm);
    node(GL_W_OUT, pp, zp);
    constexpr float SE = 0.84932180028801904272f;   // S_EX2
    P0 = s0;
    P1 = SE * s1;
    P2 = (SE * SE) * s2;
}

__device__ __forceinline__ float resp_exact32(float mf, const float4& cf, const ColG& cg) {
    return cg.A * resp_shape32(mf, cf, cg);
}
// The same with the column amplitude as a double-float A + al (al: the low part of the
// column's amplitude): one rounding per entry, and no rounding of A shared by the whole column.
__device__ __forceinline__ float resp_amp32(float mf, const float4& cf, const ColG& cg, float al) {
    const float sh = resp_shape32(mf, cf, cg);
    return fmaf(sh, al, cg.A * sh);
}

// The three node sums of the adjoint: P0 = sum w_j p_j, P1 = sum w_j t_j p_j,
// P2 = sum w_j t_j^2 p_j (t in the scaled variable, weights 8, 5, 5), same nodes as the forward.
__device__ __forceinline__ void resp_adjoint32(float mf, const float4& cf, const ColG& cg, float& P0, float& P1,
                                               float& P2) {
    float t0, tl;
    centre_df(mf, cf, cg.c_lo, t0, tl);
    const float q0 = t0 * t0;
    const float p0 = centre_node(t0, tl);
    const float z = cg.kap * t0, kk = cg.kap * INV_2LN2;
    float Sp, Sm;
    if (fabsf(z) <= 1.0f) {
        const float s = z * z, f = p0 * cg.Ck2;
        Sp = f * cosh_small(s);
        Sm = f * sinh_small(z, s);
    } else {
        outer_direct(t0, kk, Sp, Sm);
    }
    P0 = fmaf(GL_W_OUT, Sp, GL_W_MID * p0);
    P1 = fmaf(GL_W_OUT, fmaf(t0, Sp, -kk * Sm), GL_W_MID * (t0 * p0));
    P2 = fmaf(GL_W_OUT, fmaf(fmaf(kk, kk, q0), Sp, -2.0f * t0 * kk * Sm), GL_W_MID * (q0 * p0));
}

// Row recurrence of the adjoint's node sums down one column.  From row m to m + 1 the centre
// node moves by hs in the scaled variable, so
//   p0(m+1) = p0(m) rho(m),   rho(m) = 2^-(2 t0(m) hs + hs^2),   rho(m+1) = rho(m) C,  C = 2^(-2 hs^2),
// and (cosh z, sinh z) of the outer nodes (z = kap t0) rotate by the fixed step kap hs.  The
// per-column constants enter as their small parts, 1 - C and cosh(kap hs) - 1 (each from its
// series, to ~1e-10 of the constant), so a constant's FP32 rounding does not compound along
// the run: rho(m+1) = rho(m) - rho(m) (1 - C).  A run of ADJ_RUN rows starts from the exact
// evaluation of its first row (as resp_adjoint32); the FP32 recurrence error then grows about
// linearly along the run, to ~1e-6 of an entry at its end (it only enters gradient sums);
// columns narrow enough for |z| > 1 within the run take the exact form row by row.
constexpr int ADJ_RUN = 16;

struct AdjCol {
    // hs, hs^2, 1 - 2^(-2 hs^2), cosh(kap hs) - 1, sinh(kap hs), kap / (2 ln 2), 1 / Ck2
    float hs, hs2, dC, Am1, B, kk, iCk2;
};

// cosh(d) - 1 for s = d^2 <= 1 from its Taylor series through d^10 (truncation < 3e-7 of the
// result at d = 1, below 1e-20 at the d ~ 1e-2 of the bench's columns)
__device__ __forceinline__ float coshm1_small(float s) {
    float c = 2.755731922e-07f;                          // 1/10!
    c = fmaf(c, s, 2.480158730e-05f);                    // 1/8!
    c = fmaf(c, s, 1.388888889e-03f);                    // 1/6!
    c = fmaf(c, s, 4.166666667e-02f);                    // 1/4!
    c = fmaf(c, s, 0.5f);
    return c * s;
}

__device__ __forceinline__ AdjCol adj_col(const float4& cf, const ColG& cg) {
    AdjCol a;
    a.hs = cf.z;
    a.hs2 = cf.z * cf.z;
    // 1 - 2^(-x / ln 2) = 1 - e^(-x), x = 2 ln 2 hs^2: its Taylor series where x is small
    // (truncation x^6 / 720 < 3e-11 of the result for x < 0.05), else the difference
    const float x = 1.3862944f * a.hs2;
    a.dC = x < 0.05f ? x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.0f / 120.0f, -1.0f / 24.0f), 1.0f / 6.0f), -0.5f), 1.0f)
                     : 1.0f - exp2_neg(-2.0f * a.hs2);
    const float d = cg.kap * cf.z, d2 = d * d;
    a.Am1 = coshm1_small(d2);
    a.B = sinh_small(d, d2);
    a.kk = cg.kap * INV_2LN2;
    a.iCk2 = cg.Ck2 > 0.f ? 1.0f / cg.Ck2 : 0.f;
    return a;
}

// Weighted node sums of one column accumulated in a basis that needs no per-row assembly of
// the node sums: with u = p0 cosh z and v = p0 sinh z (p-+ = p0 Ck2 (cosh z -+ sinh z) / 2),
//   P0 = 5 Ck2 u + 8 p0,  P1 = 5 Ck2 (t u - kk v) + 8 t p0,
//   P2 = 5 Ck2 ((kk^2 + t^2) u - 2 kk t v) + 8 t^2 p0,
// so sum_m W P_j follows from the sums of W u, W v, W p0 and their first and second moments in
// t (AdjSums::node), and sum_m w P0 from the sums of w u and w p0.
struct AdjSums {
    float A0 = 0.f, A1 = 0.f, A2 = 0.f, B0 = 0.f, B1 = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    float Es = 0.f, Fs = 0.f, Et = 0.f, Ft = 0.f;
    __device__ __forceinline__ void add(float t, float p, float u, float v, float ws, float wt, float W) {
        const float a = W * u, b = W * v, c = W * p;
        A0 += a;
        const float ta = t * a;
        A1 += ta;
        A2 = fmaf(t, ta, A2);
        B0 += b;
        B1 = fmaf(t, b, B1);
        C0 += c;
        const float tc = t * c;
        C1 += tc;
        C2 = fmaf(t, tc, C2);
        const float sp = ws * p, tp = wt * p;
        Fs += sp;
        Es = fmaf(ws, u, Es);
        Ft += tp;
        Et = fmaf(wt, u, Et);
    }
    // (sum W P0, sum W P1, sum W P2, sum ws P0, sum wt P0) of the rows added so far
    __device__ __forceinline__ void node(float Ck2, float kk, float& p0, float& p1, float& p2, float& ps, float& pt) const {
        const float o = GL_W_OUT * Ck2;
        p0 = fmaf(o, A0, GL_W_MID * C0);
        p1 = fmaf(o, fmaf(-kk, B0, A1), GL_W_MID * C1);
        p2 = fmaf(o, fmaf(kk * kk, A0, fmaf(-2.0f * kk, B1, A2)), GL_W_MID * C2);
        ps = fmaf(o, Es, GL_W_MID * Fs);
        pt = fmaf(o, Et, GL_W_MID * Ft);
    }
};

// Adds rows mf .. mf + n - 1 (n <= ADJ_RUN) of one column into the basis sums;
// wts(k, ws, wt, W) gives row k's weights, W = ws Ssub + wt Stag + wg SA.
template <typename WF>
__device__ __forceinline__ void adj_run(float mf, int n, const float4& cf, const ColG& cg, const AdjCol& ac, WF&& wts,
                                        AdjSums& s) {
    float th, tl;
    centre_df(mf, cf, cg.c_lo, th, tl);
    const float z0 = cg.kap * th, z1 = cg.kap * fmaf((float)(ADJ_RUN - 1), ac.hs, th);
    if (fabsf(z0) <= 1.0f && fabsf(z1) <= 1.0f) {
        float p = centre_node(th, tl);
        float rho = exp2_neg(-fmaf(2.0f * th, ac.hs, ac.hs2));
        const float q = z0 * z0;
        float ch = cosh_small(q), sh = sinh_small(z0, q);
        float t = th;
#pragma unroll
        for (int k = 0; k < ADJ_RUN; ++k) {
            if (k < n) {
                float ws, wt, W;
                wts(k, ws, wt, W);
                s.add(t, p, p * ch, p * sh, ws, wt, W);
                p *= rho;
                rho = fmaf(-rho, ac.dC, rho);
                t += ac.hs;
                const float c2 = fmaf(ch, ac.Am1, fmaf(sh, ac.B, ch));
                sh = fmaf(sh, ac.Am1, fmaf(ch, ac.B, sh));
                ch = c2;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < ADJ_RUN; ++k) {
            if (k < n) {
                float ws, wt, W;
                wts(k, ws, wt, W);
                float t0, t1;
                centre_df(mf + (float)k, cf, cg.c_lo, t0, t1);
                const float p0 = centre_node(t0, t1);
                const float z = cg.kap * t0;
                float u, v;
                if (fabsf(z) <= 1.0f) {
                    const float q = z * z;
                    u = p0 * cosh_small(q);
                    v = p0 * sinh_small(z, q);
                } else {   // outer nodes directly: u = (p- + p+) / Ck2, v = (p- - p+) / Ck2
                    float Sp, Sm;
                    outer_direct(t0, ac.kk, Sp, Sm);
                    u = Sp * ac.iCk2;
                    v = Sm * ac.iCk2;
                }
                s.add(t0, p0, u, v, ws, wt, W);
            }
        }
    }
}

// The node sums P0, P1, P2 of resp_adjoint32 for rows mf .. mf + n - 1 (n <= RUN) of one
// column, by the row recurrence of adj_run from an exact start: f(k, P0, P1, P2) receives
// row mf + k.  With u = p0 cosh z, v = p0 sinh z and o = 5 Ck2,
//   P0 = o u + 8 p0,  P1 = o (t u - kk v) + 8 t p0,  P2 = o ((kk^2 + t^2) u - 2 kk t v) + 8 t^2 p0.
// Columns narrow enough for |z| > 1 within the run take resp_adjoint32 row by row.
template <int RUN = ADJ_RUN, typename F>
__device__ __forceinline__ void adj_nodes_run(float mf, int n, const float4& cf, const ColG& cg, const AdjCol& ac,
                                              F&& f) {
    float th, tl;
    centre_df(mf, cf, cg.c_lo, th, tl);
    const float z0 = cg.kap * th, z1 = cg.kap * fmaf((float)(RUN - 1), ac.hs, th);
    if (fabsf(z0) <= 1.0f && fabsf(z1) <= 1.0f) {
        float p = centre_node(th, tl);
        float rho = exp2_neg(-fmaf(2.0f * th, ac.hs, ac.hs2));
        const float q = z0 * z0;
        float ch = cosh_small(q), sh = sinh_small(z0, q);
        float t = th;
        const float o = GL_W_OUT * cg.Ck2, kk = ac.kk, kk2 = ac.kk * ac.kk;
#pragma unroll
        for (int k = 0; k < RUN; ++k) {
            if (k < n) {
                const float u = p * ch, v = p * sh, tp = t * p;
                const float P0 = fmaf(o, u, GL_W_MID * p);
                const float P1 = fmaf(o, fmaf(t, u, -kk * v), GL_W_MID * tp);
                const float P2 = fmaf(o, fmaf(fmaf(t, t, kk2), u, -2.0f * kk * t * v), GL_W_MID * (t * tp));
                f(k, P0, P1, P2);
                p *= rho;
                rho = fmaf(-rho, ac.dC, rho);
                t += ac.hs;
                const float c2 = fmaf(ch, ac.Am1, fmaf(sh, ac.B, ch));
                sh = fmaf(sh, ac.Am1, fmaf(ch, ac.B, sh));
                ch = c2;
            }
        }
    } else {
        // short runs unrolled whole, so that f may keep its rows in registers
#pragma unroll (RUN <= 8 ? RUN : 2)
        for (int k = 0; k < RUN; ++k) {
            if (k < n) {
                float P0, P1, P2;
                resp_adjoint32(mf + (float)k, cf, cg, P0, P1, P2);
                f(k, P0, P1, P2);
            }
        }
    }
}

#endif  // __CUDACC__

}  // namespace bx
