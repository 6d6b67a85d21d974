// bx_fwd_f32.cu -- Eq. 1 forward in FP32 on the CUDA cores (the mixed-precision path).
//
// Rate-first form: the Eq. 3 spectra are contracted directly,
//     lambda_h[m] = sum_i (R[m,i] / A_i) (A_i S_h[i]),   S_h[i] = sum_k r_k c_{h,k} s_k[i],
// with the column amplitude A_i folded into the spectra by k_prep32 (one rounding of the
// double-float product instead of two, and one multiply less per entry),
// and, for models with Eq. 4 terms, the response is also reduced over rows,
//     a_t[i] = sum_{m in tile t} R[m,i] Gg[m],
// from which k_mid forms every species' window marginal after pile-up.
// Unit = (row tile of TM output bins, item); 64 threads, warp q owning the two 32-row
// groups m0 + 64q + [0, 32) and m0 + 64q + [32, 64), one row of each per thread.  The warps
// never wait for each other: each stages 32 columns' parameters at a time in its own shared
// memory, lane = column, and the lanes vote three masks: the column's band touches row group
// A, row group B, and |z| <= 1 holds at every row of the warp (the generator's series branch,
// so the per-entry test is dropped).  The warp then visits only the set bits, so the work
// follows each column's own band rather than the union over the tile.
// Each thread generates the response of its bins with round-to-nearest FP32 arithmetic
// (bx_resp.cuh) and adds R S_h into Kahan-compensated accumulators at every term, so a row
// sum of ~10^3 terms keeps an error of a few roundings with no systematic sign.  For the
// column sums each lane adds R Gg of its two rows; the 32 lane values per column go through
// a padded warp-private shared buffer once per 32 columns and are stored per half tile.
// With several energy slices of the Eq. 4 terms (MES) the buffer holds R of all 64 rows and
// the column sums are formed once per slice s with its Gg_s.
#include <math.h>

#include <type_traits>

#include "bx_df.cuh"
#include "bx_internal.cuh"
#include "bx_resp.cuh"

namespace bx {

constexpr int FCH32 = 32;

// acc += a (b + bl), Kahan-compensated: bl is the low part of the column's double-float spectrum,
// so that the one rounding per term is the product's (independent from entry to entry)
__device__ __forceinline__ void kahan_fma(float& acc, float& cmp, float a, float b, float bl) {
    const float y = fmaf(a, b, fmaf(a, bl, -cmp));
    const float t = __fadd_rn(acc, y);
    cmp = __fsub_rn(__fsub_rn(t, acc), y);
    acc = t;
}

// WPC: warps per CTA, 2 (a CTA = one 128-row tile) or 1 (a CTA = one warp's 64-row half of a
// tile; the autotuner of the batched fits may pick it for small ragged items).  The warps of a
// CTA never synchronise, so the two shapes do the same work per warp.
// GC: the Gram-Charlier response (resp_shape32_gc, the toy's skewness and kurtosis terms).
template <bool TAG, bool COLS, bool MES, int WPC = 2, bool GC = false>
__global__ void __launch_bounds__(32 * WPC) k_fwd_f32(Work w) {
    // 1D item-major grid (a y dimension would cap the batch at 65535 items)
    const int unit = WPC == 2 ? (int)blockIdx.x : (int)(blockIdx.x >> 1);
    const int tile = unit % w.max_tiles, item = unit / w.max_tiles, tid = threadIdx.x;
    const Toy& T = w.toys[w.toy_of[item]];
    if (tile >= T.n_tiles || w.status[item]) return;
    const int m0 = tile * TM, M = T.M;
    const int NGRP = T.n_set > 1 ? T.n_set : 1;   // quenching groups: one column range each
    const size_t cbase = (size_t)item * w.Npad;
    const float4* colf = w.colf + cbase;
    const ColG* colg = w.colg + cbase;
    const float4* colS = w.colS32 + cbase;
    const int2* colr = w.colr + cbase;
    const int lane = tid & 31, q = WPC == 2 ? tid >> 5 : (int)(blockIdx.x & 1), g = m0 + 64 * q;
    const int qs = WPC == 2 ? q : 0;   // the warp's slot in the CTA's shared arrays
    // warp-private staging of 32 columns at a time (no block-wide barrier)
    __shared__ float4 sC[WPC][FCH32];
    __shared__ ColG sG[WPC][FCH32];
    __shared__ float4 sS[WPC][FCH32];
    // column sums: one slice -> R Gg of the lane's two rows added (32 values per column);
    // several slices (MES) -> R of each of the warp's 64 rows
    constexpr int CBR = MES ? 64 : 32;
    __shared__ float colbuf[COLS ? WPC : 1][COLS ? CBR : 1][FCH32 + 1];
    float(*cb)[FCH32 + 1] = colbuf[COLS ? qs : 0];

    const int ra = g + lane, rb = ra + 32;
    const float mfa = (float)ra, mfb = (float)rb;
    const float gga = (COLS && !MES && ra < M) ? (float)T.Gg[ra] : 0.f;
    const float ggb = (COLS && !MES && rb < M) ? (float)T.Gg[rb] : 0.f;
    const int NES = MES ? T.n_es : 1;
    __shared__ float sGg[MES ? WPC : 1][MES ? MAX_ES : 1][MES ? 64 : 1];   // Gg_s of the warp's 64 rows
    if (MES)
        for (int s = 0; s < NES; ++s) {
            sGg[qs][s][lane] = ra < M ? T.Gg32[(size_t)s * M + ra] : 0.f;
            sGg[qs][s][lane + 32] = rb < M ? T.Gg32[(size_t)s * M + rb] : 0.f;
        }
    float sa = 0.f, csa = 0.f, ta = 0.f, cta = 0.f, sb = 0.f, csb = 0.f, tb = 0.f, ctb = 0.f;
    float* apart = static_cast<float*>(w.apart) + (((size_t)item * w.max_tiles + tile) * 2 + q) * (MES ? w.nes : 1) * w.Npad;

    // one column's entries of the lane's rows: both row groups (the common case: two
    // independent chains for the scheduler) or one of them
    const float gc3 = GC ? (float)T.gc1 : 0.f, gc4 = GC ? (float)T.gc2 : 0.f;
    auto shape_t = [&](auto wide_tag, float th, float tl, const ColG& cg) {
        constexpr bool WIDE = decltype(wide_tag)::value;
        if constexpr (GC) return resp_shape32_gc_t<WIDE>(th, tl, cg, gc3, gc4);
        else return resp_shape32_t<WIDE>(th, tl, cg);
    };
    auto shape = [&](auto wide_tag, float mf, const float4& cf, const ColG& cg) {
        float th, tl;
        centre_df(mf, cf, cg.c_lo, th, tl);
        return shape_t(wide_tag, th, tl, cg);
    };
    auto column = [&](auto wide_tag, bool inA, bool inB, const float4& cf, const ColG& cg, const float4 S,
                      float& Ra, float& Rb) {
        if (inA && inB) {   // row B's centre from row A's: one double-float add
            float tha, tla, thb, tlb;
            centre_df(mfa, cf, cg.c_lo, tha, tla);
            centre_step32(tha, tla, cf, thb, tlb);
            Ra = shape_t(wide_tag, tha, tla, cg);
            Rb = shape_t(wide_tag, thb, tlb, cg);
            kahan_fma(sa, csa, Ra, S.x, S.z);
            kahan_fma(sb, csb, Rb, S.x, S.z);
            if (TAG) {
                kahan_fma(ta, cta, Ra, S.y, S.w);
                kahan_fma(tb, ctb, Rb, S.y, S.w);
            }
        } else if (inA) {
            Ra = shape(wide_tag, mfa, cf, cg);
            kahan_fma(sa, csa, Ra, S.x, S.z);
            if (TAG) kahan_fma(ta, cta, Ra, S.y, S.w);
        } else {
            Rb = shape(wide_tag, mfb, cf, cg);
            kahan_fma(sb, csb, Rb, S.x, S.z);
            if (TAG) kahan_fma(tb, ctb, Rb, S.y, S.w);
        }
    };

    for (int grp = 0; grp < NGRP; ++grp) {
    const int2 cr = tile_range(w, item, grp, tile);
    for (int c0 = cr.x; c0 < cr.y; c0 += FCH32) {
        const int ncol = min(FCH32, cr.y - c0);
        // lane = column: stage its parameters and vote, for the warp's two 32-row groups,
        // whether the column's band touches them (mA, mB) and whether |z| <= 1 at every row
        // of the warp (mW: t = (m - floor(mu/w)) hs + c is linear in the row m, so its two
        // end rows bound it)
        unsigned mA, mB, mW;
        {
            const bool in = lane < ncol;
            const int i = c0 + lane;
            const float4 cfl = in ? colf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            const ColG cgl = in ? colg[i] : ColG{0.f, 0.f, 0.f, 0.f};
            sC[qs][lane] = cfl;
            sG[qs][lane] = cgl;
            sS[qs][lane] = in ? colS[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int2 band = in ? colr[i] : make_int2(0, 0);
            const float t0 = fmaf((float)g - cfl.x, cfl.z, cfl.y), t1 = fmaf(63.0f, cfl.z, t0);
            mA = __ballot_sync(0xffffffffu, band.x < g + 32 && band.y > g);
            mB = __ballot_sync(0xffffffffu, band.x < g + 64 && band.y > g + 32);
            mW = __ballot_sync(0xffffffffu, cgl.kap * fmaxf(fabsf(t0), fabsf(t1)) <= 0.99f);
        }
        __syncwarp();
        const unsigned mAny = mA | mB;
        for (unsigned mr = mAny; mr; mr &= mr - 1u) {   // the columns whose band touches the warp
            const int c = __ffs(mr) - 1;
            const float4 cf = sC[qs][c];
            const ColG cg = sG[qs][c];
            const float4 S = sS[qs][c];
            const bool inA = (mA >> c) & 1u, inB = (mB >> c) & 1u;
            float Ra = 0.f, Rb = 0.f;
            if ((mW >> c) & 1u) column(std::true_type{}, inA, inB, cf, cg, S, Ra, Rb);
            else column(std::false_type{}, inA, inB, cf, cg, S, Ra, Rb);
            if (COLS) {
                if (MES) {
                    cb[lane][c] = Ra;
                    cb[lane + 32][c] = Rb;
                } else {
                    cb[lane][c] = fmaf(Rb, ggb, Ra * gga);
                }
            }
        }
        __syncwarp();
        if (COLS && !MES) {
            float s = 0.f;
            if ((mAny >> lane) & 1u)
                for (int j = 0; j < 32; ++j) s += cb[j][lane];
            if (lane < ncol) apart[c0 + lane] = s * sG[qs][lane].A;
            __syncwarp();
        }
        if (COLS && MES) {
            float s[MAX_ES];
#pragma unroll
            for (int e = 0; e < MAX_ES; ++e) s[e] = 0.f;
            if ((mAny >> lane) & 1u)
                for (int j = 0; j < 64; ++j) {
                    const float r = cb[j][lane];
#pragma unroll
                    for (int e = 0; e < MAX_ES; ++e)
                        if (e < NES) s[e] = fmaf(r, sGg[qs][e][j], s[e]);
                }
            if (lane < ncol)
#pragma unroll
                for (int e = 0; e < MAX_ES; ++e)
                    if (e < NES) apart[(size_t)e * w.Npad + c0 + lane] = s[e] * sG[qs][lane].A;
            __syncwarp();
        }
    }
    }
    double* lam = w.lam + (size_t)item * 2 * w.Mpad;
    if (w.lam_pairs) {   // the Kahan sum s - c as a normalised FP32 pair
        float2* lp = reinterpret_cast<float2*>(lam);
        const auto pair = [](float sum, float comp) {
            const df p = df_two_sum(sum, -comp);
            return make_float2(p.h, p.l);
        };
        if (ra < M) {
            lp[ra] = pair(sa, csa);
            if (TAG) lp[w.Mpad + ra] = pair(ta, cta);
        }
        if (rb < M) {
            lp[rb] = pair(sb, csb);
            if (TAG) lp[w.Mpad + rb] = pair(tb, ctb);
        }
        return;
    }
    if (ra < M) {
        lam[ra] = (double)sa - (double)csa;
        if (TAG) lam[w.Mpad + ra] = (double)ta - (double)cta;
    }
    if (rb < M) {
        lam[rb] = (double)sb - (double)csb;
        if (TAG) lam[w.Mpad + rb] = (double)tb - (double)ctb;
    }
}

template <int WPC, bool GC = false>
static void fwd_f32_variant(const Work& w, unsigned grid, int any_tag, int any_cols, bool mes, cudaStream_t s) {
    const unsigned g = grid * (2 / WPC);
    if (any_tag && any_cols && mes) k_fwd_f32<true, true, true, WPC, GC><<<g, 32 * WPC, 0, s>>>(w);
    else if (any_cols && mes) k_fwd_f32<false, true, true, WPC, GC><<<g, 32 * WPC, 0, s>>>(w);
    else if (any_tag && any_cols) k_fwd_f32<true, true, false, WPC, GC><<<g, 32 * WPC, 0, s>>>(w);
    else if (any_tag) k_fwd_f32<true, false, false, WPC, GC><<<g, 32 * WPC, 0, s>>>(w);
    else if (any_cols) k_fwd_f32<false, true, false, WPC, GC><<<g, 32 * WPC, 0, s>>>(w);
    else k_fwd_f32<false, false, false, WPC, GC><<<g, 32 * WPC, 0, s>>>(w);
}

cudaError_t launch_fwd_f32(const Work& w, int n, int max_tiles, int any_tag, int any_cols, cudaStream_t s) {
    const unsigned grid = (unsigned)n * (unsigned)w.max_tiles;   // decoded with w.max_tiles
    const bool mes = w.nes > 1;   // several energy slices of the Eq. 4 terms
    if (w.gc) fwd_f32_variant<2, true>(w, grid, any_tag, any_cols, mes, s);   // one tile shape for GC models
    else if (w.fwd_wpc == 1) fwd_f32_variant<1>(w, grid, any_tag, any_cols, mes, s);
    else fwd_f32_variant<2>(w, grid, any_tag, any_cols, mes, s);
    return cudaGetLastError();
}

}  // namespace bx
