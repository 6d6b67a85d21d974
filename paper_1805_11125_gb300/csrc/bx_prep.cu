// bx_prep.cu -- model set-up and the per-column stage of every evaluation.
//
// k_setup_toy (once per toy at model creation): FP32 copies of the shapes, the shapes
//   split in three (hi on a grid per species row and k-block, TF32 mid and lo) in the
//   tensor-core operand layout, FP32 pile-up spectrum,
//   and the pile-up window marginal of every energy slice W_s of the Eq. 4 terms,
//   Gg_s[m] = sum_{m' in W_s, 0 <= m'-m < L} g[m'-m] (FP64, then an FP32 copy after them).
// k_prep (FP64 model) and k_prep32 (mixed-precision modes), once per item: Eq. 1's Birks map
//   and resolution on the true-energy grid (block-wide prefix sum), the column normalisation
//   1/Phi(mu/sigma), the window masses, the rate-weighted spectra of Eq. 3 and the band limits
//   of every tile; k_prep32 also the FP32 parameters of the generated response.
#include <float.h>
#include <limits.h>
#include <math.h>

#include "bx_df.cuh"
#include "bx_internal.cuh"
#include "bx_resp.cuh"

namespace bx {

__global__ void k_setup_toy(Toy t, float* shapes32, float* shapes32l, float* S_tiles, float* g32, double* Gg) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int j = tid; j < t.K * t.N; j += nt) {
        const float h = (float)t.shapes[j];
        shapes32[j] = h;
        shapes32l[j] = (float)(t.shapes[j] - (double)h);
    }
    // species tile of k-block kb for the tensor-core forward: part p (hi | mid | lo), species
    // row n split on its own grid over the k-block (split3, from the FP64 shape: the three parts
    // hold it to ~2^-30 of the row's largest value), column c; K-major, no swizzle:
    // 8 x (4 x 4 B) core matrices, K step US * 16 B, 8-row step 128 B
    const int per_kb = 3 * US * KB;
    for (int j = tid; j < t.n_kb * US; j += nt) {
        const int kb = j / US, n = j % US;
        double v[KB];
        float mx = 0.f;
        for (int c = 0; c < KB; ++c) {
            const int i = kb * KB + c;
            v[c] = (n < t.K && i < t.N) ? t.shapes[(size_t)n * t.N + i] : 0.0;
            mx = fmaxf(mx, fabsf((float)v[c]));
        }
        const Grid g = hi_grid(mx);
        float* tile = S_tiles + (size_t)kb * per_kb;
        for (int c = 0; c < KB; ++c) {
            const float hi = rintf((float)v[c] * g.inv) * g.scale;
            const double r = v[c] - (double)hi;
            const float mid = tf32_rna((float)r);
            const float lo = tf32_rna((float)(r - (double)mid));
            const int o = (c / 4) * (US * 4) + n * 4 + (c % 4);
            tile[o] = hi;
            tile[US * KB + o] = mid;
            tile[2 * US * KB + o] = lo;
        }
    }
    for (int d = tid; d < t.L; d += nt) g32[d] = (float)t.g[d];
    for (int j = tid; j < t.n_es * t.M; j += nt) {   // one row per energy slice
        const int q = j / t.M, m = j % t.M;
        double s = 0.0;
        const int lo = max(m, t.es_lo[q]);
        const int hi = min(m + t.L - 1, t.es_hi[q] - 1);
        for (int mp = lo; mp <= hi; ++mp) s += t.g[mp - m];
        Gg[j] = s;
        reinterpret_cast<float*>(Gg + (size_t)t.n_es * t.M)[j] = (float)s;
    }
}

cudaError_t launch_setup_toy(const Toy& t, float* shapes32, float* shapes32l, float* S_tiles, float* g32, double* Gg,
                             cudaStream_t s) {
    k_setup_toy<<<152, 256, 0, s>>>(t, shapes32, shapes32l, S_tiles, g32, Gg);
    return cudaGetLastError();
}

// Upper tail Q(x) = 1 - Phi(x) = erfc(x / sqrt 2) / 2, taken as 0 from x = 9 on (Q(9) = 1.1e-19:
// below the rounding of every sum it enters; 1 - Q(x) rounds to 1 in FP64 already from x = 8.3).
constexpr double Q_CUT = 9.0;
__device__ __forceinline__ double upper_tail(double x) {
    return x >= Q_CUT ? 0.0 : 0.5 * erfc(x * 0.70710678118654752440);
}

// Gaussian mass between standard scores a < b, from the tails away from the mean.
__device__ __forceinline__ double gauss_mass(double a, double b) {
    if (a >= 0.0) return upper_tail(a) - upper_tail(b);
    if (b <= 0.0) return upper_tail(-b) - upper_tail(-a);
    return 1.0 - upper_tail(b) - upper_tail(-a);
}

// Block-wide exclusive scan of two doubles (256 threads); ta, tb receive the block totals.
__device__ void block_scan2(double& a, double& b, double& ta, double& tb, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double xa = __shfl_up_sync(0xffffffffu, ia, o), xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += xa; ib += xb; }
    }
    if (lane == 31) { sh[wid] = ia; sh[8 + wid] = ib; }
    __syncthreads();
    if (wid == 0) {
        double wa = lane < 8 ? sh[lane] : 0.0, wb = lane < 8 ? sh[8 + lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            double xa = __shfl_up_sync(0xffffffffu, wa, o), xb = __shfl_up_sync(0xffffffffu, wb, o);
            if (lane >= o) { wa += xa; wb += xb; }
        }
        if (lane < 8) { sh[16 + lane] = wa - sh[lane]; sh[24 + lane] = wb - sh[8 + lane]; }
    }
    __syncthreads();
    a = sh[16 + wid] + ia - a;
    b = sh[24 + wid] + ib - b;
    ta = sh[16 + 7] + sh[7];
    tb = sh[24 + 7] + sh[8 + 7];
    __syncthreads();
}

// One thread per true-energy column, the grid walked in chunks of 256 consecutive columns
// (coalesced loads and stores; neighbouring lanes take the same branches), the Birks prefix
// sum carried from chunk to chunk.  Tile and column-block bounds are reduced over the warp
// (redux) before one shared atomic per warp and tile.
// The FP64 model's column stage: every quantity in FP64 -- the Birks prefix sums, mu, sigma,
// 1/Phi(mu/sigma) and phi/Phi (only where mu/sigma < 9: elsewhere 1 and < 1e-18), the window
// mass (erfc only for window edges within 9 sigma), the rate-weighted spectra
// S_h[i] = sum_k r_k c_{h,k} s_k[i]; FP32 only for the response band (a work bound, not a
// result).  The FP64 generator works from mu and sigma.
template <bool MULTI>
__global__ void __launch_bounds__(256) k_prep(Work w) {
    const int item = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    if (w.skip && w.skip[item]) {   // uniform for the block: no barrier is skipped unevenly
        if (tid == 0) w.status[item] = STATUS_SKIPPED;
        return;
    }
    const Toy& T = w.toys[w.toy_of[item]];
    const int K = T.K, N = T.N, M = T.M;
    const double* th = w.theta + (size_t)item * w.tstride;
    __shared__ double sh[32];
    __shared__ int s_bad;
    __shared__ int s_tlo[MAX_SETS][MAX_TILES], s_thi[MAX_SETS][MAX_TILES], s_rlo[MAX_CB], s_rhi[MAX_CB];
    if (tid == 0) s_bad = 0;
    for (int j = tid; j < MAX_SETS * MAX_TILES; j += blockDim.x) {
        s_tlo[j / MAX_TILES][j % MAX_TILES] = INT_MAX;
        s_thi[j / MAX_TILES][j % MAX_TILES] = INT_MIN;
    }
    for (int j = tid; j < MAX_CB; j += blockDim.x) { s_rlo[j] = INT_MAX; s_rhi[j] = INT_MIN; }
    __syncthreads();
    if (tid < T.P && !isfinite(th[tid])) s_bad = 1;
    const double LY = th[K], a = th[K + 1], b = th[K + 2], c = th[K + 3], kB = th[K + 4];
    if (tid == 0 && (!(LY > 0.0) || ((T.n_rad > 0 || T.n_r2 > 0) && !(th[K + 6] > 0.0)))) s_bad = 1;

    const double w_ = T.w;
    const float wf = (float)w_, inv_wf = (float)(1.0 / w_), bandf = (float)w.band;
    const float e_min = -2.0f * wf, e_max = (M + 2.0f) * wf;
    Col64* col = w.col64 + (size_t)item * w.Npad;
    double2* cq = w.colq + (size_t)item * w.Npad;
    double2* cs = w.colS + (size_t)item * w.Npad;
    double* aW = w.aW + (size_t)item * w.nes * w.Npad;   // [nes][Npad]: one mass per energy slice
    const int NES = T.n_es;
    int2* cr = w.colr + (size_t)item * w.Npad;
    int bad = 0;
    unsigned long long inband = 0;
    // species-specific quenching: one pass per group grp of species, with Birks constant
    // kB xi[grp], into the group's columns [grp Ncs, grp Ncs + N); a position-dependent
    // response: one pass per radial shell, with light yield LY lyf[grp]
    const int NS = MULTI ? T.n_set : 1;
    for (int grp = 0; grp < NS; ++grp) {
    const int off = grp * T.Ncs;
    const double xi = MULTI ? T.xi[grp] : 1.0, kBc = kB * xi;
    const double lyf = MULTI && T.n_shell ? T.lyf[grp] : 1.0;
    double carry_x = 0.0, carry_y = 0.0;
    for (int c0 = 0; c0 < N; c0 += 256) {
        const int i = c0 + tid, ie = off + i;
        const bool in = i < N;
        // a1: Q_i = sum_{j<i} x_j + x_i / 2, x_j = dE / (1 + kB S_j); dQ_i/dkB likewise
        double x = 0.0, y = 0.0;
        if (in) {
            const double S = T.stop_pow[i], q = 1.0 + kBc * S;
            if (!(q > 0.0)) bad = 1;
            const double rq = 1.0 / q;
            x = T.dE * rq;
            y = -x * S * rq * xi;   // dx / dkB
        }
        double ex = x, ey = y, tx, ty;
        block_scan2(ex, ey, tx, ty, sh);
        int r0 = 0, r1 = 0;
        bool valid = false;
        bool live = in;
        if (MULTI && in) {   // a group's column without support: only the scan above is needed
            bool nz = false;
            for (int k = 0; k < K; ++k)
                if (set_weight<MULTI>(T, k, grp) != 0.0) nz |= T.shapes[(size_t)k * N + i] != 0.0;
            if (!nz) {
                live = false;
                col[ie] = Col64{0.0, 1.0, 0.0, 0.0};
                cq[ie] = make_double2(0.0, 0.0);
                cs[ie] = make_double2(0.0, 0.0);
                for (int q = 0; q < NES; ++q) aW[(size_t)q * w.Npad + ie] = 0.0;
                cr[ie] = make_int2(0, 0);
            }
        }
        if (live) {
            // (a radial shell's light-yield factor folded into Q: mu = LY Q, dmu/dLY = Q)
            double Q = carry_x + ex + 0.5 * x, dQ = carry_y + ey + 0.5 * y;
            if (MULTI) {
                Q *= lyf;
                dQ *= lyf;
            }
            cq[ie] = make_double2(Q, dQ);
            const double mu = LY * Q;
            const double var = fma(fma(b, mu, a), mu, c);
            const bool ok = var > 0.0;
            if (!ok) bad = 1;
            const double isig = rsqrt(fmax(var, 1e-300));
            const double sig = var * isig;
            const double z = mu * isig;
            double norm = 1.0, mills = 0.0;
            const bool gc = T.gc1 != 0.0 || T.gc2 != 0.0;
            if (z < Q_CUT) {
                // mass above 0 npe, 1 - F(-z), and the density at -z over it (d ln N / d(mu / sigma))
                double Phi = z > 0.0 ? 1.0 - upper_tail(z) : upper_tail(-z), dens = INV_SQRT_2PI * exp(-0.5 * z * z);
                if (gc) {
                    Phi += gc_cdf_term(T, -z);
                    dens *= gc_density_factor(T, -z);
                }
                norm = 1.0 / Phi;
                mills = dens * norm;
            }
            col[ie] = Col64{mu, sig, norm, mills};
            // rate-weighted spectra of the vetoed (or single) and tagged events (Eq. 3)
            double ssub = 0.0, stag = 0.0;
            bool nz = false;   // a species of this group has support in the column
            for (int k = 0; k < K; ++k) {
                const double wk = set_weight<MULTI>(T, k, grp);
                if (wk == 0.0) continue;
                nz |= T.shapes[(size_t)k * N + i] != 0.0;
                const double sk = T.shapes[(size_t)k * N + i] * th[k] * wk;
                const double t = T.tag ? T.tag[k] : 0.0;
                ssub += (T.tag ? 1.0 - t : 1.0) * sk;
                stag += t * sk;
            }
            cs[ie] = make_double2(ssub, stag);
            // mass of the column in each energy slice of the window (Eq. 4 marginals)
            for (int q = 0; q < NES; ++q) {
                const double za = (T.es_lo[q] * w_ - mu) * isig, zb = (T.es_hi[q] * w_ - mu) * isig;
                double mass = gauss_mass(za, zb);
                if (gc) mass -= gc_cdf_term(T, zb) - gc_cdf_term(T, za);
                aW[(size_t)q * w.Npad + ie] = mass * norm;
            }
            // response band: rows whose bin lies within band * sigma of mu
            const float muf = (float)mu, sigf = (float)sig;
            const float lo_e = fminf(fmaxf(muf - bandf * sigf, e_min), e_max);
            const float hi_e = fminf(fmaxf(muf + bandf * sigf, e_min), e_max);
            r0 = max(0, (int)floorf(lo_e * inv_wf));
            r1 = min(M, (int)floorf(hi_e * inv_wf) + 1);
            valid = ok && r0 < r1 && (!MULTI || nz);   // a group's columns without support are skipped
            if (valid) inband += (unsigned long long)(r1 - r0);
            cr[ie] = valid ? make_int2(r0, r1) : make_int2(0, 0);
        }
        carry_x += tx;
        carry_y += ty;
        // tile column ranges and column-block row ranges, reduced over the warp first
        const unsigned full = 0xffffffffu;
        const int t0 = valid ? r0 / TM : INT_MAX, t1 = valid ? (r1 - 1) / TM : INT_MIN;
        const int tmin = __reduce_min_sync(full, t0), tmax = __reduce_max_sync(full, t1);
        for (int t = tmin; t <= tmax; ++t) {
            const bool touch = valid && t >= t0 && t <= t1;
            const int lo = __reduce_min_sync(full, touch ? ie : INT_MAX);
            const int hi = __reduce_max_sync(full, touch ? ie + 1 : INT_MIN);
            if (lane == 0 && lo != INT_MAX) {
                atomicMin(&s_tlo[grp][t], lo);
                atomicMax(&s_thi[grp][t], hi);
            }
        }
        // a warp's 32 columns lie in one column block (BCOLS is a multiple of 32)
        const int rlo = __reduce_min_sync(full, valid ? r0 : INT_MAX);
        const int rhi = __reduce_max_sync(full, valid ? r1 : INT_MIN);
        if (lane == 0 && rlo != INT_MAX) {   // off: a multiple of BCOLS
            atomicMin(&s_rlo[ie / BCOLS], rlo);
            atomicMax(&s_rhi[ie / BCOLS], rhi);
        }
    }
    }
    // padding: the columns between groups and after the last one
    for (int i = tid; i < w.Npad; i += blockDim.x) {
        const int cpad = i / T.Ncs;
        if (cpad < NS && i - cpad * T.Ncs < N) continue;
        col[i] = Col64{0.0, 1.0, 0.0, 0.0};
        cq[i] = make_double2(0.0, 0.0);
        cs[i] = make_double2(0.0, 0.0);
        for (int q = 0; q < NES; ++q) aW[(size_t)q * w.Npad + i] = 0.0;
        cr[i] = make_int2(0, 0);
    }
    if (bad) s_bad = 1;
    if (w.count_units && inband) atomicAdd(w.units, inband);
    __syncthreads();
    for (int j = tid; j < NS * MAX_TILES; j += blockDim.x)
        w.tile_cols[(size_t)item * MAX_SETS * MAX_TILES + j] = make_int2(s_tlo[j / MAX_TILES][j % MAX_TILES],
                                                                         s_thi[j / MAX_TILES][j % MAX_TILES]);
    for (int j = tid; j < MAX_CB; j += blockDim.x)
        w.cb_rows[(size_t)item * MAX_CB + j] = make_int2(s_rlo[j], s_rhi[j]);
    if (tid == 0) w.status[item] = s_bad ? (int)BX_EDOMAIN : 0;
}

// The mixed-precision column stage takes the normalisation's Gaussian tail in FP32 from Z_F32
// standard deviations on: Q(3) = 1.3e-3, so FP32's relative error (a few 1e-7, the argument's
// rounding included) stays below 1e-9 absolute; nearer the mean it takes the FP64 tail.
constexpr float Z_F32 = 3.0f;
constexpr float INV_SQRT_2PI_F = 0.39894228f;
__device__ __forceinline__ float upper_tail32(float x) {
    return x >= (float)Q_CUT ? 0.f : 0.5f * erfcf(x * 0.70710678f);
}

// Gaussian mass of N(mu, sigma) between the npe edges e_lo < e_hi, as a double-float, from FP32
// tails on the side away from the mean: the masses enter only the Eq. 4 marginals, where an
// FP32 tail's rounding (<= ~6e-8 of the mass) averages over the several hundred columns near
// a slice's edges to ~1e-9 of a marginal bin.
__device__ __forceinline__ df slice_mass32(df e_lo, df e_hi, df mu, df isig) {
    const df zad = df_mul(df_add(e_lo, df_neg(mu)), isig), zbd = df_mul(df_add(e_hi, df_neg(mu)), isig);
    const float za = zad.h, zb = zbd.h;
    if (za <= -(float)Q_CUT && zb >= (float)Q_CUT) return df{1.f, 0.f};
    if (za >= (float)Q_CUT || zb <= -(float)Q_CUT) return df{0.f, 0.f};
    if (za >= 0.f) return df_two_sum(upper_tail32(za), -upper_tail32(zb));
    if (zb <= 0.f) return df_two_sum(upper_tail32(-zb), -upper_tail32(-za));
    return df_add(df_two_sum(1.0f, -upper_tail32(zb)), df{-upper_tail32(-za), 0.f});
}

// Block-wide exclusive scan of two double-floats (256 threads); ta, tb receive the totals.
__device__ void block_scan_df(df& a, df& b, df& ta, df& tb, float* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    df ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const df xa{__shfl_up_sync(0xffffffffu, ia.h, o), __shfl_up_sync(0xffffffffu, ia.l, o)};
        const df xb{__shfl_up_sync(0xffffffffu, ib.h, o), __shfl_up_sync(0xffffffffu, ib.l, o)};
        if (lane >= o) {
            ia = df_add(xa, ia);
            ib = df_add(xb, ib);
        }
    }
    // exclusive within the warp: the inclusive value of the previous lane
    df ea{__shfl_up_sync(0xffffffffu, ia.h, 1), __shfl_up_sync(0xffffffffu, ia.l, 1)};
    df eb{__shfl_up_sync(0xffffffffu, ib.h, 1), __shfl_up_sync(0xffffffffu, ib.l, 1)};
    if (lane == 0) ea = eb = df{0.f, 0.f};
    if (lane == 31) {
        sh[4 * wid] = ia.h; sh[4 * wid + 1] = ia.l; sh[4 * wid + 2] = ib.h; sh[4 * wid + 3] = ib.l;
    }
    __syncthreads();
    if (wid == 0) {
        df wa = lane < 8 ? df{sh[4 * lane], sh[4 * lane + 1]} : df{0.f, 0.f};
        df wb = lane < 8 ? df{sh[4 * lane + 2], sh[4 * lane + 3]} : df{0.f, 0.f};
        const df oa = wa, ob = wb;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const df xa{__shfl_up_sync(0xffffffffu, wa.h, o), __shfl_up_sync(0xffffffffu, wa.l, o)};
            const df xb{__shfl_up_sync(0xffffffffu, wb.h, o), __shfl_up_sync(0xffffffffu, wb.l, o)};
            if (lane >= o) {
                wa = df_add(xa, wa);
                wb = df_add(xb, wb);
            }
        }
        if (lane < 8) {   // exclusive warp prefixes at 32.., totals at 64..
            const df pa = df_add(wa, df_neg(oa)), pb = df_add(wb, df_neg(ob));
            sh[32 + 4 * lane] = pa.h; sh[33 + 4 * lane] = pa.l; sh[34 + 4 * lane] = pb.h; sh[35 + 4 * lane] = pb.l;
        }
        if (lane == 7) { sh[64] = wa.h; sh[65] = wa.l; sh[66] = wb.h; sh[67] = wb.l; }
    }
    __syncthreads();
    a = df_add(df{sh[32 + 4 * wid], sh[33 + 4 * wid]}, ea);
    b = df_add(df{sh[34 + 4 * wid], sh[35 + 4 * wid]}, eb);
    ta = df{sh[64], sh[65]};
    tb = df{sh[66], sh[67]};
    __syncthreads();
}

// The per-column stage of the mixed-precision modes in double-float FP32 (bx_df.cuh, ~2^-44
// relative): the Birks prefix sums, 1/(1 + kB S), mu, sigma^2, 1/sigma by one Newton step, the
// generator's split constants.  FP64 only where a column's Gaussian reaches 0 npe within
// Z_F32 = 3 sigma (1/Phi, phi/Phi; FP32 tails beyond) and for the FP64 copies of mu, sigma, Q,
// dQ/dkB that the adjoint's chain rule reads (formed on the integer pipe, f2d).  The window
// masses come from FP32 tails and go out as FP32 pairs.
// SHELL: the sets are the radial shells of a position-dependent response (every species in every
// set with its fraction, a light-yield factor per set) instead of quenching groups.
template <bool MULTI, bool GC = false, bool SHELL = false>
__global__ void __launch_bounds__(256, 3) k_prep32(Work w) {
    const int item = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    if (w.skip && w.skip[item]) {
        if (tid == 0) w.status[item] = STATUS_SKIPPED;
        return;
    }
    const Toy& T = w.toys[w.toy_of[item]];
    const int K = T.K, N = T.N, M = T.M;
    const double* th = w.theta + (size_t)item * w.tstride;
    __shared__ float sh[72];
    __shared__ int s_bad;
    __shared__ int s_tlo[MAX_SETS][MAX_TILES], s_thi[MAX_SETS][MAX_TILES], s_rlo[MAX_CB], s_rhi[MAX_CB];
    // rates times the tag fractions (vetoed, tagged) as FP32 pairs, per set of columns times the
    // species' weight in the set (0 outside its quenching group, its fraction in a radial shell)
    constexpr int NSR = MULTI ? MAX_SETS : 1;
    __shared__ float s_rate[NSR][4][KMAX];
    __shared__ df s_par[10 + MAX_ES];   // LY, a, b, c, kB, dE, w S_EX2, 1/w, A's constant factor, slice edges
    if (tid == 0) s_bad = 0;
    for (int j = tid; j < MAX_SETS * MAX_TILES; j += blockDim.x) {
        s_tlo[j / MAX_TILES][j % MAX_TILES] = INT_MAX;
        s_thi[j / MAX_TILES][j % MAX_TILES] = INT_MIN;
    }
    for (int j = tid; j < MAX_CB; j += blockDim.x) { s_rlo[j] = INT_MAX; s_rhi[j] = INT_MIN; }
    if (tid < NSR * KMAX) {
        const int k = tid % KMAX, c = tid / KMAX;
        double rs = 0.0, rt = 0.0;
        if (k < K && (!MULTI || c < T.n_set)) {
            const double t = T.tag ? T.tag[k] : 0.0, wk = (SHELL ? T.shw[c][k] : set_weight<MULTI>(T, k, c));
            rs = th[k] * (T.tag ? 1.0 - t : 1.0) * wk;
            rt = th[k] * t * wk;
        }
        const float rsh = (float)rs, rth = (float)rt;
        s_rate[c][0][k] = rsh;
        s_rate[c][1][k] = (float)(rs - (double)rsh);
        s_rate[c][2][k] = rth;
        s_rate[c][3][k] = (float)(rt - (double)rth);
    }
    if (tid < 10 + T.n_es) {   // edges of the energy slices (npe): e_q = es_lo[q], e_S = es_hi[S - 1]
        const int q = tid - 9;
        const double v = tid < 5    ? th[K + tid]
                         : tid == 5 ? T.dE
                         : tid == 6 ? T.w * S_EX2
                         : tid == 7 ? 1.0 / T.w
                         : tid == 8 ? 0.5 * INV_SQRT_2PI * GL_W_SCALE * T.w
                                    : (q < T.n_es ? T.es_lo[q] : T.es_hi[T.n_es - 1]) * T.w;
        s_par[tid] = df_from(v);
    }
    __syncthreads();
    if (tid < T.P && !isfinite(th[tid])) s_bad = 1;
    if (tid == 0 && (!(th[K] > 0.0) || ((T.n_rad > 0 || T.n_r2 > 0) && !(th[K + 6] > 0.0)))) s_bad = 1;
    const df LY = s_par[0], pa = s_par[1], pb = s_par[2], pc = s_par[3], kB = s_par[4], dE = s_par[5];
    const df wS = s_par[6], iw = s_par[7], cAw = s_par[8];
    const int NES = T.n_es;
    const double w_ = T.w;
    const float wf = (float)w_, inv_wf = iw.h, bandf = (float)w.band;
    const float e_min = -2.0f * wf, e_max = (M + 2.0f) * wf;
    Col64* col = w.col64 + (size_t)item * w.Npad;
    double2* cq = w.colq + (size_t)item * w.Npad;
    float4* cf = w.colf + (size_t)item * w.Npad;
    ColG* cg = w.colg + (size_t)item * w.Npad;
    float4* cs32 = w.colS32 + (size_t)item * w.Npad;
    float* cAl = w.colAl + (size_t)item * w.Npad;
    float2* aW2 = reinterpret_cast<float2*>(w.aW + (size_t)item * w.nes * w.Npad);   // [nes][Npad] FP32 pairs
    int2* cr = w.colr + (size_t)item * w.Npad;
    const df gln{0.38729834f, (float)(0.38729833462074170 - (double)0.38729834f)};   // sqrt(3/5) / 2
    const df ln2d{0.6931471824645996f, -1.9046542121259336e-09f};                      // ln 2
    const df ln4{1.3862944f, (float)(1.3862943611198906 - (double)1.3862944f)};      // 2 ln 2
    int bad = 0;
    unsigned long long inband = 0;
    // species-specific quenching: one pass per group grp of species, with Birks constant
    // kB xi[grp], into the group's columns [grp Ncs, grp Ncs + N)
    const int NS = MULTI ? T.n_set : 1;
    for (int grp = 0; grp < NS; ++grp) {
    const int off = grp * T.Ncs;
    constexpr bool shell = MULTI && SHELL;   // a radial shell: light yield LY lyf[grp]
    const df lyf = shell ? df_from(T.lyf[grp]) : df{1.f, 0.f};
    const df xid = MULTI ? df_from(T.xi[grp]) : df{1.f, 0.f};
    const df kBc = MULTI ? df_mul(kB, xid) : kB;
    df carry_x{0.f, 0.f}, carry_y{0.f, 0.f};
    for (int c0 = 0; c0 < N; c0 += 256) {
        const int i = c0 + tid, ie = off + i;
        const bool in = i < N;
        df S{0.f, 0.f}, x{0.f, 0.f}, y{0.f, 0.f};
        if (in) {
            if (T.stop32) {
                const float2 s2 = T.stop32[i];
                S = df{s2.x, s2.y};
            } else {
                S = df_from(T.stop_pow[i]);
            }
            const df q = df_addf(df_mul(kBc, S), 1.0f);
            if (!(q.h > 0.f)) bad = 1;
            const df rq = df_recip(q);
            x = df_mul(dE, rq);
            y = df_neg(df_mul(df_mul(x, S), rq));   // dx / d(kB xi)
            if (MULTI) y = df_mul(y, xid);            // dx / dkB
        }
        df ex = x, ey = y, tx, ty;
        block_scan_df(ex, ey, tx, ty, sh);
        int r0 = 0, r1 = 0;
        bool valid = false;
        bool live = in;
        // a quenching group's column without support: only the scan above is needed (radial
        // shells carry every species: their columns without support are dropped after the
        // spectra below, like any other)
        if (MULTI && !shell && in) {
            bool nz = false;
            for (int k = 0; k < K; ++k)
                if (T.set_of[k] == grp) nz |= T.shapes[(size_t)k * N + i] != 0.0;
            if (!nz) {
                live = false;
                col[ie] = Col64{0.0, 1.0, 0.0, 0.0};
                cq[ie] = make_double2(0.0, 0.0);
                cf[ie] = make_float4(0.f, 0.f, 0.f, 0.f);
                cg[ie] = ColG{0.f, 0.f, 0.f, 0.f};
                cs32[ie] = make_float4(0.f, 0.f, 0.f, 0.f);
                cAl[ie] = 0.f;
                for (int q = 0; q < NES; ++q) aW2[(size_t)q * w.Npad + ie] = make_float2(0.f, 0.f);
                cr[ie] = make_int2(0, 0);
            }
        }
        if (live) {
            df Q = df_add(df_add(carry_x, ex), df{0.5f * x.h, 0.5f * x.l});
            df dQ = df_add(df_add(carry_y, ey), df{0.5f * y.h, 0.5f * y.l});
            if (shell) {   // the shell's light-yield factor folded into Q: mu = LY Q, dmu/dLY = Q
                Q = df_mul(Q, lyf);
                dQ = df_mul(dQ, lyf);
            }
            cq[ie] = make_double2(df_to_double(Q), df_to_double(dQ));
            const df mu = df_mul(LY, Q);
            const df var = df_add(df_mul(df_add(df_mul(pb, mu), pa), mu), pc);
            const bool ok = var.h > 0.f;
            if (!ok) bad = 1;
            const df isig = df_rsqrt(ok ? var : df{1.f, 0.f});
            const df sig = df_mul(var, isig);
            const df z = df_mul(mu, isig);
            const double mud = df_to_double(mu), sigd = df_to_double(sig);
            double norm = 1.0, mills = 0.0;
            df normd{1.f, 0.f};
            const bool gc = GC && (T.gc1 != 0.0 || T.gc2 != 0.0);   // Gram-Charlier: FP64 to Q_CUT (its terms)
            if (z.h < Z_F32 || (gc && z.h < (float)Q_CUT)) {
                const double zd = df_to_double(z);
                double Phi = zd > 0.0 ? 1.0 - upper_tail(zd) : upper_tail(-zd), dens = INV_SQRT_2PI * exp(-0.5 * zd * zd);
                if (gc) {
                    Phi += gc_cdf_term(T, -zd);
                    dens *= gc_density_factor(T, -zd);
                }
                norm = 1.0 / Phi;
                mills = dens * norm;
                normd = df_from(norm);
            } else if (z.h < (float)Q_CUT) {   // Q(z) <= 1.3e-3
                const float q = upper_tail32(z.h), qn = q / (1.0f - q);
                normd = df_fast(1.0f, qn);
                norm = df_to_double(normd);
                mills = f2d(INV_SQRT_2PI_F * exp2f(-0.72134752f * df_mul(z, z).h) * (1.0f + qn));
            }
            col[ie] = Col64{mud, sigd, norm, mills};
            // generator constants: t0 = (m + 1/2 - mu/w) hs = (m - jf) hs + c
            const df u = df_mul(mu, iw);
            float jf = floorf(u.h);
            if (u.h == jf && u.l < 0.f) jf -= 1.0f;
            const df frac = df_addf(u, -jf);
            const df hs = df_mul(wS, isig);
            const df cc = df_mul(df_addf(df_neg(frac), 0.5f), hs);
            cf[ie] = make_float4(jf, cc.h, hs.h, hs.l);
            const df kk = df_mul(gln, hs), kq = df_mul(kk, kk);
            // Ck2 = 2 2^(-kk^2) as a double-float: for kk^2 ln2 < 1/100 from the series of e^(-x)
            // through x^4 (truncation < 1e-12), else FP32.  The forward multiplies by its FP32 value
            // Ck2.h; the error Ck2.l, the same at every row of the column, is folded into the column
            // amplitude: R / A = 8 p0 + 5 Ck2 p0 cosh z, with cosh z = 1 + O(1e-2) over the band,
            // so A (8 + 5 Ck2) / (8 + 5 Ck2.h) leaves ~1e-2 Ck2.l of it.
            df Ck2;
            {
                const df x = df_mul(kq, ln2d);
                if (x.h < 0.01f) {
                    const float x2 = x.h * x.h;
                    const float tail = x2 * fmaf(x.h, fmaf(x.h, 1.0f / 24.0f, -1.0f / 6.0f), 0.5f);
                    Ck2 = df_addf(df_neg(x), 1.0f);
                    Ck2 = df_addf(Ck2, tail);
                    Ck2 = df{2.0f * Ck2.h, 2.0f * Ck2.l};
                } else {
                    Ck2 = df{2.0f * exp2_neg(-kq.h, -kq.l), 0.0f};
                }
            }
            const df Ad0 = df_mul(df_mul(cAw, isig), normd);
            const float node_w = fmaf(GL_W_OUT, Ck2.h, GL_W_MID);   // 8 + 5 Ck2.h
            const df Ad = df_mul(Ad0, df_fast(1.0f, GL_W_OUT * Ck2.l / node_w));
            cg[ie] = ColG{df_mul(ln4, kk).h, Ck2.h, cc.l, Ad.h};
            cAl[ie] = Ad.l;
            // rate-weighted spectra of the vetoed (or single) and tagged events (Eq. 3) in
            // double-float from the split shapes and rates, times the column amplitude A (the FP32
            // forward generates R / A); kept as double-float pairs, so that no rounding of a
            // column's spectrum (shared by every row of its band) reaches the expected counts
            bool nz = false;   // a species of this group has support in the column
            df ss{0.f, 0.f}, st{0.f, 0.f};
            if (T.shapes32) {   // the model's split copy: four species' loads in flight at a time
                for (int k0 = 0; k0 < K; k0 += 4) {
                    float hv[4], lv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = k0 + q;
                        const bool use = k < K && (!MULTI || (SHELL ? T.shw[grp][k] != 0.0 : T.set_of[k] == grp));
                        hv[q] = use ? T.shapes32[(size_t)k * N + i] : 0.f;
                        lv[q] = use ? T.shapes32l[(size_t)k * N + i] : 0.f;
                    }
                    const float(&rg)[4][KMAX] = s_rate[MULTI ? grp : 0];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (hv[q] == 0.f) continue;
                        const int k = k0 + q;
                        const df sk{hv[q], lv[q]};
                        nz = true;
                        ss = df_add(ss, df_mul(df{rg[0][k], rg[1][k]}, sk));
                        st = df_add(st, df_mul(df{rg[2][k], rg[3][k]}, sk));
                    }
                }
            } else {            // a descriptor with FP64 shapes only
                const float(&rg)[4][KMAX] = s_rate[MULTI ? grp : 0];
                for (int k = 0; k < K; ++k) {
                    if (MULTI && (SHELL ? T.shw[grp][k] == 0.0 : T.set_of[k] != grp)) continue;
                    const double x = T.shapes[(size_t)k * N + i];
                    if (x == 0.0) continue;
                    const df sk = df_from(x);
                    nz = true;
                    ss = df_add(ss, df_mul(df{rg[0][k], rg[1][k]}, sk));
                    st = df_add(st, df_mul(df{rg[2][k], rg[3][k]}, sk));
                }
            }
            const df As = df_mul(Ad, ss), At = df_mul(Ad, st);
            cs32[ie] = make_float4(As.h, At.h, As.l, At.l);
            // slice masses times 1/Phi, as FP32 pairs
            for (int q = 0; q < NES; ++q) {   // one mass per energy slice
                df aw;
                if (gc) {   // Gram-Charlier: the mass in FP64 from the CDF F = Phi - phi C
                    const double mudd = df_to_double(mu), isd = df_to_double(isig);
                    const double za = (df_to_double(s_par[9 + q]) - mudd) * isd, zb = (df_to_double(s_par[10 + q]) - mudd) * isd;
                    aw = df_from((gauss_mass(za, zb) - (gc_cdf_term(T, zb) - gc_cdf_term(T, za))) * norm);
                } else {
                    aw = df_mul(slice_mass32(s_par[9 + q], s_par[10 + q], mu, isig), normd);
                }
                aW2[(size_t)q * w.Npad + ie] = make_float2(aw.h, aw.l);
            }
            // response band
            const float lo_e = fminf(fmaxf(mu.h - bandf * sig.h, e_min), e_max);
            const float hi_e = fminf(fmaxf(mu.h + bandf * sig.h, e_min), e_max);
            r0 = max(0, (int)floorf(lo_e * inv_wf));
            r1 = min(M, (int)floorf(hi_e * inv_wf) + 1);
            valid = ok && r0 < r1 && (!MULTI || nz);   // a group's columns without support are skipped
            if (valid) inband += (unsigned long long)(r1 - r0);
            cr[ie] = valid ? make_int2(r0, r1) : make_int2(0, 0);
        }
        carry_x = df_add(carry_x, tx);
        carry_y = df_add(carry_y, ty);
        const unsigned full = 0xffffffffu;
        const int t0 = valid ? r0 / TM : INT_MAX, t1 = valid ? (r1 - 1) / TM : INT_MIN;
        const int tmin = __reduce_min_sync(full, t0), tmax = __reduce_max_sync(full, t1);
        for (int t = tmin; t <= tmax; ++t) {
            const bool touch = valid && t >= t0 && t <= t1;
            const int lo = __reduce_min_sync(full, touch ? ie : INT_MAX);
            const int hi = __reduce_max_sync(full, touch ? ie + 1 : INT_MIN);
            if (lane == 0 && lo != INT_MAX) {
                atomicMin(&s_tlo[grp][t], lo);
                atomicMax(&s_thi[grp][t], hi);
            }
        }
        const int rlo = __reduce_min_sync(full, valid ? r0 : INT_MAX);
        const int rhi = __reduce_max_sync(full, valid ? r1 : INT_MIN);
        if (lane == 0 && rlo != INT_MAX) {   // a warp's 32 columns lie in one block (off: a multiple of BCOLS)
            atomicMin(&s_rlo[ie / BCOLS], rlo);
            atomicMax(&s_rhi[ie / BCOLS], rhi);
        }
    }
    }
    // padding: the columns between groups and after the last one
    for (int i = tid; i < w.Npad; i += blockDim.x) {
        const int cpad = i / T.Ncs;
        if (cpad < NS && i - cpad * T.Ncs < N) continue;
        col[i] = Col64{0.0, 1.0, 0.0, 0.0};
        cq[i] = make_double2(0.0, 0.0);
        cf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        cg[i] = ColG{0.f, 0.f, 0.f, 0.f};
        cs32[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        cAl[i] = 0.f;
        for (int q = 0; q < NES; ++q) aW2[(size_t)q * w.Npad + i] = make_float2(0.f, 0.f);
        cr[i] = make_int2(0, 0);
    }
    if (bad) s_bad = 1;
    if (w.count_units && inband) atomicAdd(w.units, inband);
    __syncthreads();
    for (int j = tid; j < NS * MAX_TILES; j += blockDim.x)
        w.tile_cols[(size_t)item * MAX_SETS * MAX_TILES + j] = make_int2(s_tlo[j / MAX_TILES][j % MAX_TILES],
                                                                         s_thi[j / MAX_TILES][j % MAX_TILES]);
    for (int j = tid; j < MAX_CB; j += blockDim.x)
        w.cb_rows[(size_t)item * MAX_CB + j] = make_int2(s_rlo[j], s_rhi[j]);
    if (tid == 0) w.status[item] = s_bad ? (int)BX_EDOMAIN : 0;
}

cudaError_t launch_prep(const Work& w, int n, cudaStream_t s) {
    if (w.precision == BX_FP64) {
        if (w.multi_set) k_prep<true><<<n, 256, 0, s>>>(w);
        else k_prep<false><<<n, 256, 0, s>>>(w);
    } else {
        if (w.shells) {   // radial shells of the response (their own instantiations)
            if (w.gc) k_prep32<true, true, true><<<n, 256, 0, s>>>(w);
            else k_prep32<true, false, true><<<n, 256, 0, s>>>(w);
        } else if (w.gc) {
            if (w.multi_set) k_prep32<true, true><<<n, 256, 0, s>>>(w);
            else k_prep32<false, true><<<n, 256, 0, s>>>(w);
        } else if (w.multi_set) k_prep32<true><<<n, 256, 0, s>>>(w);
        else k_prep32<false><<<n, 256, 0, s>>>(w);
    }
    return cudaGetLastError();
}

}  // namespace bx
