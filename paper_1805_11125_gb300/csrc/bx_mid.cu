// bx_mid.cu -- per-item assembly of the likelihood from the forward reductions.
//
// One CTA per item.  Inputs: the Eq. 3 spectra lambda_h[m] (rate-first forward) or the
// species spectra v[m][k] (tensor-core forward, lambda_h = sum_k r_k c_{h,k} v_k), with
// h = TFC-vetoed (c = 1 - t_k) and TFC-tagged (c = t_k), or one spectrum (c = 1);
//   Eq. 2  mu_h = (1 - eps) lambda_h + eps (g * lambda_h) on the window (direct sum,
//          compensated when it runs in FP32);
//   Eq. 4  A_k = r_k c_{vetoed,k} sum_m v_k[m] G_W[m], G_W = (1 - eps) 1_W + eps Gg: the
//          expected vetoed events of species k in the window after pile-up (rate-first:
//          sum_m v_k G_W = sum_i s_k[i] ((1 - eps) aW[i] + eps a[i]), with the closed-form
//          window mass aW[i] and the forward's column sums a[i]); radial bins
//          sum_k A_k p_k[rho] (closed-form shell integrals) and pulse-shape bins
//          sum_k A_k q_k[j]; with several energy slices W_s of the window, one such
//          marginal, radial and pulse-shape histogram per slice (G_W,s, aW_s, a_s);
//   -lnL   sum of mu - n + n log1p((n - mu)/mu): the terms in FP64, or for the
//          mixed-precision modes in a cancellation-free FP32 form where mu/2 <= n <= 2 mu
//          and in double-float elsewhere; the sum in FP64 with Neumaier compensation inside
//          each thread (k_mid32: compensated FP32) and TwoSum-style merging across the block.
// With want_grad it also writes the adjoint inputs of the response stage: per row the
// pile-up-correlated residual weights wt_h[m] and G_W[m], per species the coefficients
// that turn them into dNLL/dR[m,i], and the gradient of eps, s_r and the parts of the
// rate gradient that do not pass through the response (the rest comes from k_bwd_*).
#include <math.h>

#include "bx_df.cuh"
#include "bx_internal.cuh"

namespace bx {

constexpr int MID_THREADS = 512;
constexpr int MID_WARPS = MID_THREADS / 32;

// Sum NV per-thread doubles over the block; result in out[0..NV) (all threads see it).
template <int NV>
__device__ void block_sum(double (&x)[NV], double* red, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const double s = warp_sum(x[j]);
        if (lane == 0) red[wid * NV + j] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NV; j += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < MID_WARPS; ++q) s += red[q * NV + j];
        out[j] = s;
    }
    __syncthreads();
}

// Dot product acc += a b over a long, decaying sequence.  In FP32 the terms that fall below
// half an ulp of the accumulator would all be rounded away, a one-sided loss of the pile-up
// tail (-2e-8 relative in mu for a 400-bin kernel); Kahan compensation keeps them.
struct Dot32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float y = fmaf(a, b, -c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
struct Dot64 {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <typename TV> struct DotT { using type = Dot64; };
template <> struct DotT<float> { using type = Dot32; };

// bc_term_far on FP64 arguments (the TF32X3 assembly)
__device__ __forceinline__ bool bc_term_far_d(double n, double mu, double& term, double& wb) {
    df t;
    float wf;
    if (!bc_term_far(df_from(n), df_from(mu), t, wf)) return false;
    term = df_to_double(t);
    wb = (double)wf;
    return true;
}

// Radial bin probabilities of the Eq. 4 marginal: internal events uniform in volume,
// external ones exponential in depth from r_iv (attenuation length att_len s_r), with the
// shell integrals at the nrad + 1 bin edges and at r = 0 taken once each.  Called by the whole
// block (one barrier inside).
__device__ void radial_probs(const Toy& T, double s_r, double* sF, double* sdF, double* pint, double* pext,
                             double* dpext) {
    const int nrad = T.n_rad;
    const double lamA = T.att_len * s_r;
    for (int e = threadIdx.x; e <= nrad + 1; e += blockDim.x) {
        const double r = e < nrad ? T.r_fid * e / nrad : (e == nrad ? T.r_fid : 0.0);
        shell_F(r, T.r_iv, lamA, sF[e], sdF[e]);
    }
    __syncthreads();
    const double tot = sF[nrad] - sF[nrad + 1], dtot = sdF[nrad] - sdF[nrad + 1];
    for (int b = threadIdx.x; b < nrad; b += blockDim.x) {
        const double ra = T.r_fid * b / nrad, rb = T.r_fid * (b + 1) / nrad;
        pint[b] = (rb * rb * rb - ra * ra * ra) / (T.r_fid * T.r_fid * T.r_fid);
        const double p = (sF[b + 1] - sF[b]) / tot;
        pext[b] = p;
        dpext[b] = ((sdF[b + 1] - sdF[b]) / tot - p * dtot / tot) * T.att_len;
    }
}

template <typename TV, bool SPECIES>
__global__ void __launch_bounds__(MID_THREADS, (sizeof(TV) == sizeof(float) && !SPECIES) ? 2 : 1)
    k_mid(Work w, int want_grad, int want_mu) {
    extern __shared__ __align__(16) double dsm[];
    const int item = blockIdx.x, tid = threadIdx.x;
    const Toy& T = w.toys[w.toy_of[item]];
    const int K = T.K, M = T.M, nw = T.nw, m_lo = T.m_lo, L = T.L, H = T.has_tag ? 2 : 1;
    const int nrad = T.n_rad, npsd = T.n_psd, nb = T.nb, NES = T.n_es;   // NES = 1 in the species mode
    const int nradS = NES * nrad, npsdS = NES * npsd;                    // bins of all energy slices
    double* gmid = w.gmid + (size_t)item * PMAX;
    if (w.status[item]) {
        if (tid == 0) w.nll[item] = INFINITY;
        if (tid < PMAX) gmid[tid] = 0.0;
        return;
    }
    const double* th = w.theta + (size_t)item * w.tstride;
    const double eps = th[K + 5], s_r = th[K + 6];
    const TV* v = static_cast<const TV*>(w.v) + (size_t)item * w.Mpad * US;
    const size_t vlo = (size_t)w.cap * w.Mpad * US;   // offset of the lo plane of v

    double* lam = dsm;                                  // [H][M]
    double* muw = lam + 2 * M;                          // [H][nw]
    TV* lamT = reinterpret_cast<TV*>(muw + 2 * nw);     // [H][M], reused for wt after the pile-up
    TV* puT = lamT + 2 * M;                             // [H][nw] pile-up convolution part
    TV* wvT = puT + 2 * nw;                             // [H][nw] 1 - n/mu
    TV* gT = wvT + 2 * nw;                              // [L]

    // per energy slice q: s_SA[q][k] = sum v_k G_W,q, s_SA[q][KMAX + k] its d/deps; s_beta[q][k]
    __shared__ double s_rs[KMAX], s_rt[KMAX], s_SA[MAX_ES][2 * KMAX], s_beta[MAX_ES][KMAX], s_gr[2 * KMAX];
    __shared__ double s_aint[MAX_ES], s_aext[MAX_ES];
    __shared__ double s_pint[MAX_RAD], s_pext[MAX_RAD], s_dpext[MAX_RAD], s_mur[MAX_RAD], s_wr[MAX_RAD];
    __shared__ double s_F[MAX_RAD + 2], s_dF[MAX_RAD + 2];
    __shared__ double s_mup[MAX_PSD], s_wp[MAX_PSD];
    __shared__ double red[MID_WARPS * 2 * KMAX];
    __shared__ double s_misc[8];
    __shared__ int s_dom;

    if (tid == 0) s_dom = 0;
    if (tid < K) {
        const double r = th[tid], t = T.tag ? T.tag[tid] : 0.0;
        s_rs[tid] = r * (T.tag ? 1.0 - t : 1.0);
        s_rt[tid] = r * t;
    }
    for (int d = tid; d < L; d += MID_THREADS) gT[d] = (TV)T.g[d];
    __syncthreads();

    // Eq. 3: the energy spectra on the full axis
    constexpr bool species = SPECIES;
    const double* lamg = w.lam + (size_t)item * 2 * w.Mpad;
    for (int m = tid; m < M; m += MID_THREADS) {
        double ls = 0.0, lt = 0.0;
        if (species) {
            const TV* vr = v + (size_t)m * US;
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) {
                    const double x = (double)vr[k] + (double)vr[vlo + k];
                    ls += s_rs[k] * x;
                    lt += s_rt[k] * x;
                }
        } else {
            ls = lamg[m];
            lt = H == 2 ? lamg[w.Mpad + m] : 0.0;
        }
        lam[m] = ls;
        lamT[m] = (TV)ls;
        if (H == 2) {
            lam[M + m] = lt;
            lamT[M + m] = (TV)lt;
        }
    }
    __syncthreads();

    // Eq. 2 on the window
    for (int idx = tid; idx < H * nw; idx += MID_THREADS) {
        const int h = idx / nw, j = idx % nw, m = m_lo + j;
        const TV* x = lamT + h * M;
        const int dmax = min(m, L - 1);
        typename DotT<TV>::type conv;
        for (int d = 0; d <= dmax; ++d) conv.add(gT[d], x[m - d]);
        const double cv = conv.value();
        puT[idx] = (TV)cv;
        muw[idx] = (1.0 - eps) * lam[h * M + m] + eps * cv;
    }

    // Eq. 4: window marginals of the vetoed species spectra after pile-up
    const bool mv = nrad > 0 || npsd > 0;
    for (int qs = 0; mv && qs < NES; ++qs) {   // one pass per energy slice
        double part[2 * KMAX];
#pragma unroll
        for (int k = 0; k < 2 * KMAX; ++k) part[k] = 0.0;
        if (species) {
            for (int m = tid; m < M; m += MID_THREADS) {
                const double inW = m >= T.es_lo[qs] && m < T.es_hi[qs] ? 1.0 : 0.0, gg = T.Gg[(size_t)qs * M + m];
                const double GW = (1.0 - eps) * inW + eps * gg, dG = gg - inW;
                const TV* vr = v + (size_t)m * US;
#pragma unroll
                for (int k = 0; k < KMAX; ++k)
                    if (k < K) {
                        const double x = (double)vr[k] + (double)vr[vlo + k];
                        part[k] += x * GW;
                        part[KMAX + k] += x * dG;
                    }
            }
        } else {
            // sum_m v_k[m] G_W[m] = sum_i s_k[i] ((1 - eps) aW[i] + eps a[i]), a[i] from the
            // per-tile column sums of the forward (valid on each tile's band only)
            constexpr int HALF = sizeof(TV) == sizeof(float) ? 2 : 1;   // slots per tile
            const TV* ap = static_cast<const TV*>(w.apart) + (size_t)item * w.max_tiles * HALF * w.nes * w.Npad;
            const double* aWi = w.aW + ((size_t)item * w.nes + qs) * w.Npad;
            const int lane = tid & 31, wid = tid >> 5;
            {   // FP64 model (the rate-first FP32 mode runs k_mid32)
                // column ie = grp Ncs + i of quenching group grp carries the species of that group
                // (of radial shell grp: every species, with its fraction in the shell)
                for (int ie = tid; ie < T.Next; ie += MID_THREADS) {
                    const int grp = ie / T.Ncs, i = ie - grp * T.Ncs;
                    if (i >= T.N) continue;
                    const int2* tcols = w.tile_cols + ((size_t)item * MAX_SETS + grp) * MAX_TILES;
                    double ag = 0.0;
                    for (int t = 0; t < T.n_tiles; ++t) {
                        const int2 cr = tcols[t];
                        if (ie >= cr.x && ie < cr.y)
                            for (int h = 0; h < HALF; ++h) ag += (double)ap[(((size_t)t * HALF + h) * w.nes + qs) * w.Npad + ie];
                    }
                    const double aw = aWi[ie];
                    const double GW = (1.0 - eps) * aw + eps * ag, dG = ag - aw;
#pragma unroll
                    for (int k = 0; k < KMAX; ++k)
                        if (k < K) {
                            const double wk = set_weight<true>(T, k, grp);
                            if (wk == 0.0) continue;
                            const double x = T.shapes[(size_t)k * T.N + i] * wk;
                            part[k] += x * GW;
                            part[KMAX + k] += x * dG;
                        }
                }
#pragma unroll
                for (int k = 0; k < 2 * KMAX; ++k) {
                    const double r = warp_sum(part[k]);
                    if (lane == 0) red[wid * 2 * KMAX + k] = r;
                }
            }
            __syncthreads();
            if (tid < 2 * KMAX) {
                double v = 0.0;
                for (int q = 0; q < MID_WARPS; ++q) v += red[q * 2 * KMAX + tid];
                s_SA[qs][tid] = v;
            }
            __syncthreads();
        }
        // s_SA[q][k] = sum v G_W,q, s_SA[q][KMAX+k] = sum v dG_W,q/deps
        if (species) block_sum<2 * KMAX>(part, red, s_SA[qs]);
    }
    // radial bin probabilities (internal: uniform in volume; external: exponential from r_iv)
    if (nrad > 0) radial_probs(T, s_r, s_F, s_dF, s_pint, s_pext, s_dpext);
    __syncthreads();
    if (mv && tid < NES) {   // internal and external vetoed events of slice tid
        double aint = 0.0, aext = 0.0;
        for (int k = 0; k < K; ++k) {
            const double A = s_rs[k] * s_SA[tid][k];
            if (nrad > 0 && T.rad_class[k] == BX_RAD_EXTERNAL) aext += A; else aint += A;
        }
        s_aint[tid] = aint;
        s_aext[tid] = aext;
    }
    __syncthreads();
    for (int b = tid; b < nradS; b += MID_THREADS) {
        const int q = b / nrad, r = b - q * nrad;
        s_mur[b] = s_aint[q] * s_pint[r] + s_aext[q] * s_pext[r];
    }
    for (int j = tid; j < npsdS; j += MID_THREADS) {
        const int q = j / npsd, r = j - q * npsd;
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += s_rs[k] * s_SA[q][k] * T.psd[(size_t)k * npsd + r];
        s_mup[j] = s;
    }
    __syncthreads();

    // -lnL over every bin
    Neu acc{0.0, 0.0};
    double geps = 0.0;
    int dom = 0;
    const int nwin = H * nw;
    for (int b = tid; b < nb; b += MID_THREADS) {
        const double n = T.cnt[b];
        double mu;
        if (b < nwin) mu = muw[b];
        else if (b < nwin + nradS) mu = s_mur[b - nwin];
        else mu = s_mup[b - nwin - nradS];
        double term, wb = 1.0;
        if (n == 0.0) term = mu;
        else if (!(mu > 0.0 && isfinite(mu))) { dom = 1; term = 0.0; }
        else if (sizeof(TV) == sizeof(float) && bc_term_far_d(n, mu, term, wb)) {}
        else {
            term = (mu - n) + n * log1p((n - mu) / mu);
            wb = 1.0 - n / mu;
        }
        neu_add(acc, term);
        if (want_mu) w.mu[(size_t)item * w.nbmax + b] = mu;
        if (want_grad) {
            if (b < nwin) {
                const int h = b / nw, j = b % nw;
                wvT[b] = (TV)wb;
                geps += wb * ((double)puT[b] - lam[h * M + m_lo + j]);
            } else if (b < nwin + nradS) s_wr[b - nwin] = wb;
            else s_wp[b - nwin - nradS] = wb;
        }
    }
    // merge the compensated partial sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Neu other{__shfl_xor_sync(0xffffffffu, acc.s, o), __shfl_xor_sync(0xffffffffu, acc.c, o)};
        acc = neu_merge(acc, other);
        geps += __shfl_xor_sync(0xffffffffu, geps, o);
    }
    if (dom) s_dom = 1;
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) {
        red[wid * 3 + 0] = acc.s;
        red[wid * 3 + 1] = acc.c;
        red[wid * 3 + 2] = geps;
    }
    __syncthreads();
    if (tid == 0) {
        Neu tot{0.0, 0.0};
        double ge = 0.0;
        for (int q = 0; q < MID_WARPS; ++q) {
            tot = neu_merge(tot, Neu{red[q * 3], red[q * 3 + 1]});
            ge += red[q * 3 + 2];
        }
        w.nll[item] = s_dom ? INFINITY : tot.s + tot.c;
        if (s_dom) w.status[item] = BX_EDOMAIN;
        s_misc[2] = ge;
    }
    __syncthreads();
    if (!want_grad || s_dom) {
        if (tid < PMAX) gmid[tid] = 0.0;
        return;
    }

    // ---- adjoint inputs
    // beta_q,k = dNLL/dA_k^(q) = sum_rho w_rad,q p_k[rho] + sum_j w_psd,q q_k[j], per energy slice q
    if (mv) {
        for (int qk = wid; qk < NES * K; qk += MID_WARPS) {
            const int q = qk / K, k = qk - q * K;
            double s = 0.0;
            const bool ext = nrad > 0 && T.rad_class[k] == BX_RAD_EXTERNAL;
            for (int b = lane; b < nrad; b += 32) s += s_wr[q * nrad + b] * (ext ? s_pext[b] : s_pint[b]);
            for (int j = lane; j < npsd; j += 32) s += s_wp[q * npsd + j] * T.psd[(size_t)k * npsd + j];
            s = warp_sum(s);
            if (lane == 0) s_beta[q][k] = s;
        }
    }
    __syncthreads();
    // pile-up-correlated weights wt_h[m] (adjoint of Eq. 2) and G_W[m], written per row
    TV* rowW = static_cast<TV*>(w.rowW) + (size_t)item * (2 + w.nes) * w.Mpad;
    TV* wt = lamT;   // lambda copies are no longer needed
    for (int idx = tid; idx < H * M; idx += MID_THREADS) {
        const int h = idx / M, m = idx % M;
        const TV* wh = wvT + h * nw;
        const int d0 = max(0, m_lo - m), d1 = min(L - 1, M - 1 - m);
        typename DotT<TV>::type acc;
        for (int d = d0; d <= d1; ++d) acc.add(gT[d], wh[m + d - m_lo]);
        const double direct = (m >= m_lo) ? (1.0 - eps) * (double)wh[m - m_lo] : 0.0;
        const TV val = (TV)(direct + eps * acc.value());
        wt[idx] = val;
        rowW[(size_t)h * w.Mpad + m] = val;
    }
    for (int j = tid; j < w.nes * M; j += MID_THREADS) {   // G_W,q[m] of every slice q (0 beyond the toy's)
        const int q = j / M, m = j - q * M;
        if (q == 0 && H == 1) rowW[(size_t)w.Mpad + m] = (TV)0;
        const double inW = q < NES && m >= T.es_lo[q] && m < T.es_hi[q] ? 1.0 : 0.0;
        rowW[(size_t)(2 + q) * w.Mpad + m] =
            mv && q < NES ? (TV)((1.0 - eps) * inW + eps * T.Gg[(size_t)q * M + m]) : (TV)0;
    }
    __syncthreads();
    // rate gradient, part through the spectra: sum_h c_{h,k} sum_m wt_h[m] v_k[m]; only the
    // tensor-core path has v here, the rate-first path gets it from k_bwd_* as
    // sum_h c_{h,k} sum_i s_k[i] sum_m R[m,i] wt_h[m]
    if (species) {
        double part[2 * KMAX];
#pragma unroll
        for (int k = 0; k < 2 * KMAX; ++k) part[k] = 0.0;
        for (int m = tid; m < M; m += MID_THREADS) {
            const double a0 = (double)wt[m], a1 = H == 2 ? (double)wt[M + m] : 0.0;
            const TV* vr = v + (size_t)m * US;
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) {
                    const double x = (double)vr[k] + (double)vr[vlo + k];
                    part[k] += a0 * x;
                    part[KMAX + k] += a1 * x;
                }
        }
        block_sum<2 * KMAX>(part, red, s_gr);
    } else if (tid < 2 * KMAX) {
        s_gr[tid] = 0.0;
    }
    __syncthreads();
    double* coef = w.coef + (size_t)item * (2 + w.nes) * KMAX;
    if (tid < K) {
        const int k = tid;
        const double t = T.tag ? T.tag[k] : 0.0, csub = T.tag ? 1.0 - t : 1.0;
        double gk = csub * s_gr[k] + (H == 2 ? t * s_gr[KMAX + k] : 0.0);
        for (int q = 0; mv && q < NES; ++q) gk += s_beta[q][k] * csub * s_SA[q][k];
        gmid[k] = gk;
        coef[k] = s_rs[k];
        coef[KMAX + k] = s_rt[k];
    }
    if (tid >= K && tid < KMAX) {
        coef[tid] = 0.0;
        coef[KMAX + tid] = 0.0;
    }
    for (int j = tid; j < w.nes * KMAX; j += MID_THREADS) {
        const int q = j / KMAX, k = j - q * KMAX;
        coef[(size_t)(2 + q) * KMAX + k] = mv && q < NES && k < K ? s_beta[q][k] * s_rs[k] : 0.0;
    }
    if (tid == 0) {
        double ge = s_misc[2];
        for (int q = 0; mv && q < NES; ++q)
            for (int k = 0; k < K; ++k) ge += s_beta[q][k] * s_rs[k] * s_SA[q][KMAX + k];
        double gs = 0.0;
        for (int b = 0; b < nradS; ++b) gs += s_wr[b] * s_aext[b / nrad] * s_dpext[b % nrad];
        for (int j = K; j < K + 5; ++j) gmid[j] = 0.0;
        gmid[K + 5] = ge;
        gmid[K + 6] = gs;
        for (int j = K + 7; j < PMAX; ++j) gmid[j] = 0.0;
    }
}

// Register-blocked pile-up sums: PR consecutive outputs per thread, g read four taps at a
// time, a sliding window of the other operand in registers.  Plain FP32 partial sums over 32
// taps are folded into a Kahan pair: the partials are of the size of their terms, so no tail
// term falls below the accumulator's rounding (the one-sided loss a plain running sum has).
constexpr int PR = 4;
constexpr int PBLK = 8;   // chunks of PR taps per partial sum
struct Kahan4 {
    float s[PR], c[PR], p[PR];
    __device__ __forceinline__ Kahan4() {
#pragma unroll
        for (int j = 0; j < PR; ++j) s[j] = c[j] = p[j] = 0.f;
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int j = 0; j < PR; ++j) {
            const float y = __fsub_rn(p[j], c[j]);
            const float t = __fadd_rn(s[j], y);
            c[j] = __fsub_rn(__fsub_rn(t, s[j]), y);
            s[j] = t;
            p[j] = 0.f;
        }
    }
    __device__ __forceinline__ float value(int j) const { return __fsub_rn(s[j], c[j]); }
};

// Convolution out_j = sum_{d < dend} g[d] x[base + j - d], j < PR.  g: 16-byte aligned, zero
// from L up to a multiple of PR; x readable (zero) from base - dend - 10 to base + PR - 1, and
// x + base - 7 16-byte aligned (the four values entering per PR taps come as one float4).
__device__ __forceinline__ void conv_block(const float* g, const float* x, int base, int dend, Kahan4& k) {
    float xw[2 * PR - 1];   // xw[t] = x[base - d0 - 3 + t]
#pragma unroll
    for (int t = 0; t < 2 * PR - 1; ++t) xw[t] = x[base - 3 + t];
    int cnt = 0;
    for (int d0 = 0; d0 < dend; d0 += PR) {
        const float4 g4 = *reinterpret_cast<const float4*>(g + d0);
        const float gg[PR] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
        for (int t = 0; t < PR; ++t)
#pragma unroll
            for (int j = 0; j < PR; ++j) k.p[j] = fmaf(gg[t], xw[3 + j - t], k.p[j]);
#pragma unroll
        for (int t = 2 * PR - 2; t >= PR; --t) xw[t] = xw[t - PR];
        const float4 xn = *reinterpret_cast<const float4*>(x + base - d0 - 7);   // 16-byte aligned (mid32_padl)
        xw[0] = xn.x;
        xw[1] = xn.y;
        xw[2] = xn.z;
        xw[3] = xn.w;
        if (++cnt == PBLK) {
            k.fold();
            cnt = 0;
        }
    }
    k.fold();
}

// Correlation out_j = sum_{d0s <= d < dend} g[d] y[base + j + d], j < PR, d0s a multiple of
// PR.  y readable (zero) from base + d0s to base + dend + 9, y + base + 7 16-byte aligned.
__device__ __forceinline__ void corr_block(const float* g, const float* y, int base, int d0s, int dend, Kahan4& k) {
    float yw[2 * PR - 1];   // yw[t] = y[base + d0 + t]
#pragma unroll
    for (int t = 0; t < 2 * PR - 1; ++t) yw[t] = y[base + d0s + t];
    int cnt = 0;
    for (int d0 = d0s; d0 < dend; d0 += PR) {
        const float4 g4 = *reinterpret_cast<const float4*>(g + d0);
        const float gg[PR] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
        for (int t = 0; t < PR; ++t)
#pragma unroll
            for (int j = 0; j < PR; ++j) k.p[j] = fmaf(gg[t], yw[j + t], k.p[j]);
#pragma unroll
        for (int t = 0; t < PR - 1; ++t) yw[t] = yw[t + PR];
        const float4 yn = *reinterpret_cast<const float4*>(y + base + d0 + 2 * PR - 1);   // aligned (mid32_padw)
        yw[PR - 1] = yn.x;
        yw[PR] = yn.y;
        yw[PR + 1] = yn.z;
        yw[PR + 2] = yn.w;
        if (++cnt == PBLK) {
            k.fold();
            cnt = 0;
        }
    }
    k.fold();
}

// Zero padding of the pile-up operands in shared memory
// (at least 16 / 8 before each lambda / weight row, chosen by the item's m_lo so that the window
// values conv_block and corr_block fetch per four taps start on a 16-byte boundary; rows of a
// multiple of four floats, at least 4 / 16 zeros after)
__host__ __device__ constexpr int mid32_padl(int m_lo) { return 16 + ((7 - m_lo) & 3); }
__host__ __device__ constexpr int mid32_padw(int m_lo) { return 8 + ((m_lo + 1) & 3); }
__host__ __device__ constexpr int mid32_lrow(int M) { return (19 + M + 4 + 3) & ~3; }
__host__ __device__ constexpr int mid32_wrow(int nw) { return (11 + nw + 16 + 3) & ~3; }
__host__ __device__ constexpr int mid32_gn(int L) { return ((L + PR - 1) / PR) * PR + PR; }
__host__ __device__ constexpr int mid32_pun(int nw) { return (2 * nw + 3) & ~3; }   // the [2][nw] pile-up part

// Baker-Cousins term from double-float n and mu in double-float (bc_term_far: ln(n/mu) to
// ~2e-11, so a term's absolute error is ~2e-11 n |n/mu - 1|); the term goes into a compensated
// FP32 sum, wb = 1 - n/mu.  (An FP32 form of the term, relative error ~1e-7, let the terms of a
// few hundred at points far from the optimum add up to |Delta(-2 lnL)| ~ 1e-3 over 1900 bins.)
__device__ __forceinline__ void bc_term_df(df n, df mu, Sum32& acc, float& wb) {
    df t;
    if (!bc_term_far(n, mu, t, wb)) {   // n/mu beyond [1e-30, 1e30]: FP64
        const double nd = df_to_double(n), md = df_to_double(mu);
        t = df_from((md - nd) + nd * log1p((nd - md) / md));
        wb = (float)(1.0 - nd / md);
    }
    acc.add(t.h);
    acc.c = __fadd_rn(acc.c, t.l);
}

// The assembly of the rate-first mixed-precision mode (BX_FP32): the quantities of k_mid with
// every per-bin and per-column step in FP32 or double-float FP32 (value hi + lo, ~2^-44
// relative) instead of FP64, GB300's FP64 rate being 1/64 of its FP32 rate.  The forward
// hands over lambda_h as FP32 pairs, the column stage the window masses aW; -lnL is a
// compensated FP32 sum (TwoSum per term, merged across the block in FP64).  FP64 remains for
// the radial and pulse-shape marginals (one value per bin, ~100 bins).
// MES: several energy slices of the Eq. 4 terms (otherwise one, with compile-time strides).
template <bool MES>
__global__ void __launch_bounds__(MID_THREADS, 2) k_mid32(Work w, int want_grad, int want_mu) {
    extern __shared__ __align__(16) double dsm[];
    const int item = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const Toy& T = w.toys[w.toy_of[item]];
    const int K = T.K, M = T.M, nw = T.nw, m_lo = T.m_lo, L = T.L, H = T.has_tag ? 2 : 1;
    const int nrad = T.n_rad, npsd = T.n_psd, nb = T.nb, NES = MES ? T.n_es : 1;
    const int WNES = MES ? w.nes : 1;   // slice stride of the workspace
    const int nradS = NES * nrad, npsdS = NES * npsd;   // bins of all energy slices
    double* gmid = w.gmid + (size_t)item * PMAX;
    if (w.status[item]) {
        if (tid == 0) w.nll[item] = INFINITY;
        if (tid < PMAX) gmid[tid] = 0.0;
        return;
    }
    const double* th = w.theta + (size_t)item * w.tstride;
    const double eps = th[K + 5], s_r = th[K + 6];
    __shared__ float s_eps[4];   // eps and 1 - eps as FP32 pairs
    if (tid == 0) {
        const df e = df_from(eps), o = df_from(1.0 - eps);
        s_eps[0] = e.h; s_eps[1] = e.l; s_eps[2] = o.h; s_eps[3] = o.l;
    }
    const float2* lamg = reinterpret_cast<const float2*>(w.lam + (size_t)item * 2 * w.Mpad);

    const int lrow = mid32_lrow(M), wrow = mid32_wrow(nw), gn = mid32_gn(L);
    const int padl = mid32_padl(m_lo), padw = mid32_padw(m_lo);
    float2* muw = reinterpret_cast<float2*>(dsm);          // [H][nw] mu as FP32 pairs
    float* gT = reinterpret_cast<float*>(muw + 2 * nw);     // [gn] g, zero-padded (16-byte aligned)
    float* lamP = gT + gn;                                  // [H][lrow] FP32 lambda, zero-padded
    float* puT = lamP + 2 * lrow;                           // [H][nw] pile-up convolution part
    float* wvP = puT + mid32_pun(nw);                       // [H][wrow] 1 - n/mu, zero-padded (16-byte aligned)
    float2* colGW = reinterpret_cast<float2*>(wvP + 2 * wrow);   // [Next] G_W per column (8-byte aligned)
    float* coldG = reinterpret_cast<float*>(colGW + T.Next);     // [Next] dG_W/deps per column

    // per energy slice q: s_SA[q][k] = sum v_k G_W,q, s_SA[q][KMAX + k] its d/deps; s_beta[q][k]
    constexpr int XS = MES ? MAX_ES : 1;
    __shared__ double s_rs[KMAX], s_rt[KMAX], s_SA[XS][2 * KMAX], s_beta[XS][KMAX];
    __shared__ double s_aint[XS], s_aext[XS];
    __shared__ double s_pint[MAX_RAD], s_pext[MAX_RAD], s_dpext[MAX_RAD], s_mur[MAX_RAD], s_wr[MAX_RAD];
    __shared__ double s_F[MAX_RAD + 2], s_dF[MAX_RAD + 2];
    __shared__ double s_mup[MAX_PSD], s_wp[MAX_PSD];
    __shared__ double red[MID_WARPS * 2 * KMAX];
    __shared__ double s_misc[8];
    __shared__ int s_dom;

    if (tid == 0) s_dom = 0;
    if (tid < K) {
        const double r = th[tid], t = T.tag ? T.tag[tid] : 0.0;
        s_rs[tid] = r * (T.tag ? 1.0 - t : 1.0);
        s_rt[tid] = r * t;
    }
    for (int d = tid; d < gn; d += MID_THREADS) gT[d] = d < L ? T.g32[d] : 0.f;
    for (int q = tid; q < 2 * lrow; q += MID_THREADS) {
        const int h = q / lrow, m = q % lrow - padl;
        lamP[q] = (h < H && m >= 0 && m < M) ? lamg[(size_t)h * w.Mpad + m].x : 0.f;
    }
    for (int q = tid; q < 2 * wrow; q += MID_THREADS) wvP[q] = 0.f;
    __syncthreads();
    const df epsd{s_eps[0], s_eps[1]}, omed{s_eps[2], s_eps[3]};
    const float epsf = epsd.h, omef = omed.h;

    // Eq. 2 on the window: mu = (1 - eps) lambda + eps (g * lambda), the convolution in
    // compensated FP32 (conv_block), the mix in double-float
    const int ngw = (nw + PR - 1) / PR;
    for (int q = tid; q < H * ngw; q += MID_THREADS) {
        const int h = q / ngw, j0 = (q % ngw) * PR, m0 = m_lo + j0;
        Kahan4 k;
        conv_block(gT, lamP + h * lrow + padl, m0, min(L, m0 + PR), k);
#pragma unroll
        for (int j = 0; j < PR; ++j)
            if (j0 + j < nw) {
                const float cv = k.value(j);
                puT[h * nw + j0 + j] = cv;
                const float2 l2 = lamg[(size_t)h * w.Mpad + m0 + j];
                const df mu = df_add(df_mul(omed, df{l2.x, l2.y}), df_mulf(epsd, cv));
                muw[h * nw + j0 + j] = make_float2(mu.h, mu.l);
            }
    }

    // Eq. 4: sum_m v_k[m] G_W[m] = sum_i s_k[i] ((1 - eps) aW[i] + eps a[i]), a[i] from the
    // per-tile column sums of the forward (valid on each tile's band only).  G_W per column
    // first (double-float), then one warp per species, its lanes splitting the columns;
    // products and sums in compensated FP32 (TwoProduct, TwoSum): the terms are non-negative
    // and the result is the exact sum to a few 1e-15 of its size.
    const bool mv = nrad > 0 || npsd > 0;
    // one pass per energy slice q (its own masses aW_q and column sums a_q), the per-column
    // buffers reused
    for (int qs = 0; mv && qs < NES; ++qs) {
        const float* ap = static_cast<const float*>(w.apart) + (size_t)item * w.max_tiles * 2 * WNES * w.Npad;
        const float2* aW2 = reinterpret_cast<const float2*>(w.aW + ((size_t)item * WNES + qs) * w.Npad);
        for (int i = tid; i < T.Next; i += MID_THREADS) {   // every column of every quenching group
            const int2* tcols = w.tile_cols + ((size_t)item * MAX_SETS + (T.n_set > 1 ? i / T.Ncs : 0)) * MAX_TILES;
            float agf = 0.f;   // a few positive terms; enters G_W with weight eps
            for (int t = 0; t < T.n_tiles; ++t) {
                const int2 cr = tcols[t];
                if (i >= cr.x && i < cr.y)
                    agf += ap[(((size_t)t * 2) * WNES + qs) * w.Npad + i] + ap[(((size_t)t * 2 + 1) * WNES + qs) * w.Npad + i];
            }
            const float2 a2 = aW2[i];
            const df aw{a2.x, a2.y};
            // G_W = aW + eps (a - aW): eps (a - aW) in FP32 is ~5e-9 of G_W
            const float dG = df_addf(df_neg(aw), agf).h;
            const df GW = df_addf(aw, epsf * dG);
            colGW[i] = make_float2(GW.h, GW.l);
            coldG[i] = dG;
        }
        __syncthreads();
        for (int k = wid; k < K; k += MID_WARPS) {
            const float* sk = T.shapes32 + (size_t)k * T.N;
            // the columns of k's quenching group, or of every radial shell (weighted in FP64 by the
            // species' fraction of events in the shell)
            const int c_lo = T.n_shell ? 0 : (T.n_set > 1 ? T.set_of[k] : 0);
            const int c_hi = T.n_shell ? T.n_set : c_lo + 1;
            double A0 = 0.0, A1 = 0.0;
            for (int c = c_lo; c < c_hi; ++c) {
                const double wk = T.n_shell ? T.shw[c][k] : 1.0;
                if (wk == 0.0) continue;
                const int off = c * T.Ncs;
                Sum32 a0, a1;
                for (int i = lane; i < T.N; i += 32) {
                    const float x = sk[i];
                    const float2 g2 = colGW[off + i];
                    a0.add_prod(x, g2.x, g2.y);
                    a1.add_prod(x, coldG[off + i], 0.f);
                }
                a0 = a0.warp_reduce();
                a1 = a1.warp_reduce();
                A0 += wk * ((double)a0.s + (double)a0.c);
                A1 += wk * ((double)a1.s + (double)a1.c);
            }
            if (lane == 0) {   // s_SA[q][k] = sum v G_W,q, s_SA[q][KMAX + k] = sum v dG_W,q/deps
                s_SA[qs][k] = A0;
                s_SA[qs][KMAX + k] = A1;
            }
        }
        __syncthreads();   // colGW, coldG are reused by the next slice
    }
    // radial bin probabilities (internal: uniform in volume; external: exponential from r_iv)
    if (nrad > 0) radial_probs(T, s_r, s_F, s_dF, s_pint, s_pext, s_dpext);
    __syncthreads();
    if (mv && tid < NES) {   // internal and external vetoed events of slice tid
        double aint = 0.0, aext = 0.0;
        for (int k = 0; k < K; ++k) {
            const double A = s_rs[k] * s_SA[tid][k];
            if (nrad > 0 && T.rad_class[k] == BX_RAD_EXTERNAL) aext += A; else aint += A;
        }
        s_aint[tid] = aint;
        s_aext[tid] = aext;
    }
    __syncthreads();
    for (int b = tid; b < nradS; b += MID_THREADS) {
        const int q = MES ? b / nrad : 0, r = b - q * nrad;
        s_mur[b] = s_aint[q] * s_pint[r] + s_aext[q] * s_pext[r];
    }
    for (int j = tid; j < npsdS; j += MID_THREADS) {
        const int q = MES ? j / npsd : 0, r = j - q * npsd;
        double v = 0.0;
        for (int k = 0; k < K; ++k) v += s_rs[k] * s_SA[q][k] * T.psd[(size_t)k * npsd + r];
        s_mup[j] = v;
    }
    __syncthreads();

    // -lnL over every bin
    Sum32 acc;
    float geps = 0.f;
    int dom = 0;
    const int nwin = H * nw;
    for (int b = tid; b < nb; b += MID_THREADS) {
        const float2 n2 = T.cnt32[b];
        const df n{n2.x, n2.y};
        df mu;
        if (b < nwin) {
            const float2 m2 = muw[b];
            mu = df{m2.x, m2.y};
        } else {
            mu = df_from(b < nwin + nradS ? s_mur[b - nwin] : s_mup[b - nwin - nradS]);
        }
        float wb = 1.0f;
        if (n.h == 0.f) {
            acc.add(mu.h);
            acc.c = __fadd_rn(acc.c, mu.l);
        } else if (!(mu.h > 0.f && isfinite(mu.h))) {
            dom = 1;
        } else {
            bc_term_df(n, mu, acc, wb);
        }
        if (want_mu) w.mu[(size_t)item * w.nbmax + b] = df_to_double(mu);
        if (want_grad) {
            if (b < nwin) {
                const int h = b / nw, j = b % nw;
                wvP[h * wrow + padw + j] = wb;
                geps = fmaf(wb, puT[b] - lamP[h * lrow + padl + m_lo + j], geps);
            } else if (b < nwin + nradS) s_wr[b - nwin] = (double)wb;
            else s_wp[b - nwin - nradS] = (double)wb;
        }
    }
    acc = acc.warp_reduce();
    geps = warp_sum(geps);
    if (dom) s_dom = 1;
    if (lane == 0) {
        red[wid * 3 + 0] = (double)acc.s;
        red[wid * 3 + 1] = (double)acc.c;
        red[wid * 3 + 2] = (double)geps;
    }
    __syncthreads();
    if (tid == 0) {
        Neu tot{0.0, 0.0};
        double ge = 0.0;
        for (int q = 0; q < MID_WARPS; ++q) {
            tot = neu_merge(tot, Neu{red[q * 3], red[q * 3 + 1]});
            ge += red[q * 3 + 2];
        }
        w.nll[item] = s_dom ? INFINITY : tot.s + tot.c;
        if (s_dom) w.status[item] = BX_EDOMAIN;
        s_misc[2] = ge;
    }
    __syncthreads();
    if (!want_grad || s_dom) {
        if (tid < PMAX) gmid[tid] = 0.0;
        return;
    }

    // ---- adjoint inputs
    // beta_q,k = dNLL/dA_k^(q) = sum_rho w_rad,q p_k[rho] + sum_j w_psd,q q_k[j], per energy slice q
    if (mv) {
        for (int qk = wid; qk < NES * K; qk += MID_WARPS) {
            const int q = MES ? qk / K : 0, k = qk - q * K;
            double v = 0.0;
            const bool ext = nrad > 0 && T.rad_class[k] == BX_RAD_EXTERNAL;
            for (int b = lane; b < nrad; b += 32) v += s_wr[q * nrad + b] * (ext ? s_pext[b] : s_pint[b]);
            for (int j = lane; j < npsd; j += 32) v += s_wp[q * npsd + j] * T.psd[(size_t)k * npsd + j];
            v = warp_sum(v);
            if (lane == 0) s_beta[q][k] = v;
        }
    }
    __syncthreads();
    // pile-up-correlated weights wt_h[m] (adjoint of Eq. 2) and G_W[m], per row, in FP32:
    // wt_h[m] = (1 - eps) w_h[m] [m in W] + eps sum_d g[d] w_h[m + d]
    float* rowW = static_cast<float*>(w.rowW) + (size_t)item * (2 + WNES) * w.Mpad;
    const int ngm = (M + PR - 1) / PR;
    for (int q = tid; q < H * ngm; q += MID_THREADS) {
        const int h = q / ngm, m0 = (q % ngm) * PR, base = m0 - m_lo;   // window index at d = 0
        const int d0s = max(0, -(base + PR - 1)) / PR * PR, dend = min(L, nw - base);
        const float* wh = wvP + h * wrow + padw;
        Kahan4 k;
        if (dend > d0s) corr_block(gT, wh, base, d0s, dend, k);
#pragma unroll
        for (int j = 0; j < PR; ++j) {
            const int m = m0 + j;
            if (m < M) {
                const float direct = m >= m_lo ? omef * wh[m - m_lo] : 0.f;
                rowW[(size_t)h * w.Mpad + m] = fmaf(epsf, k.value(j), direct);
            }
        }
    }
    for (int j = tid; j < WNES * M; j += MID_THREADS) {   // G_W,q[m] of every slice q (0 beyond the toy's)
        const int q = MES ? j / M : 0, m = j - q * M;
        if (q == 0 && H == 1) rowW[(size_t)w.Mpad + m] = 0.f;
        rowW[(size_t)(2 + q) * w.Mpad + m] =
            mv && q < NES ? fmaf(epsf, T.Gg32[(size_t)q * M + m], m >= T.es_lo[q] && m < T.es_hi[q] ? omef : 0.f) : 0.f;
    }
    // the rate gradient through the spectra comes from the adjoint kernel
    double* coef = w.coef + (size_t)item * (2 + WNES) * KMAX;
    if (tid < K) {
        const int k = tid;
        const double csub = T.tag ? 1.0 - T.tag[k] : 1.0;
        double gk = 0.0;
        for (int q = 0; mv && q < NES; ++q) gk += s_beta[q][k] * csub * s_SA[q][k];
        gmid[k] = gk;
        coef[k] = s_rs[k];
        coef[KMAX + k] = s_rt[k];
    }
    if (tid >= K && tid < KMAX) {
        coef[tid] = 0.0;
        coef[KMAX + tid] = 0.0;
    }
    for (int j = tid; j < WNES * KMAX; j += MID_THREADS) {
        const int q = MES ? j / KMAX : 0, k = j - q * KMAX;
        coef[(size_t)(2 + q) * KMAX + k] = mv && q < NES && k < K ? s_beta[q][k] * s_rs[k] : 0.0;
    }
    if (tid == 0) {
        double ge = s_misc[2];
        for (int q = 0; mv && q < NES; ++q)
            for (int k = 0; k < K; ++k) ge += s_beta[q][k] * s_rs[k] * s_SA[q][KMAX + k];
        double gs = 0.0;
        for (int b = 0; b < nradS; ++b) {
            const int q = MES ? b / nrad : 0;
            gs += s_wr[b] * s_aext[q] * s_dpext[b - q * nrad];
        }
        for (int j = K; j < K + 5; ++j) gmid[j] = 0.0;
        gmid[K + 5] = ge;
        gmid[K + 6] = gs;
        for (int j = K + 7; j < PMAX; ++j) gmid[j] = 0.0;
    }
}

template <typename TV, bool SPECIES>
static cudaError_t launch_mid_t(const Work& w, int n, size_t smem, int want_grad, int want_mu, cudaStream_t s) {
    // the attribute is set once per size (outside any stream capture that replays it)
    static size_t set = 0;
    if (smem > set) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_mid<TV, SPECIES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set = smem;
    }
    k_mid<TV, SPECIES><<<n, MID_THREADS, smem, s>>>(w, want_grad, want_mu);
    return cudaGetLastError();
}

// Dynamic shared memory of the assembly kernel the workspace's precision selects, for the
// model's largest axis (Mmax), window (nwmax) and pile-up spectrum (Lmax).
static size_t mid_dynamic_smem(const Work& w, int Mmax, int nwmax, int Lmax) {
    if (w.precision != BX_FP32) {   // k_mid: lambda and mu in FP64, the rest in the kernel's type
        const size_t tv = w.precision == BX_FP64 ? sizeof(double) : sizeof(float);
        return (size_t)(2 * Mmax + 2 * nwmax) * sizeof(double) + (size_t)(2 * Mmax + 4 * nwmax + Lmax) * tv + 64;
    }
    // k_mid32: mu pairs [2][nw], g, lambda rows, pile-up part [2][nw], weight rows (zero-padded),
    // G_W and dG_W/deps per column
    return (size_t)2 * nwmax * sizeof(float2) +
           (size_t)(mid32_gn(Lmax) + 2 * mid32_lrow(Mmax) + mid32_pun(nwmax) + 2 * mid32_wrow(nwmax)) * sizeof(float) +
           (size_t)w.Npad * (sizeof(float2) + sizeof(float));
}

cudaError_t mid_smem_budget(const Work& w, int Mmax, int nwmax, int Lmax, size_t* need, size_t* avail) {
    *need = mid_dynamic_smem(w, Mmax, nwmax, Lmax);
    cudaFuncAttributes fa{};
    cudaError_t e;
    if (w.precision == BX_FP64) e = cudaFuncGetAttributes(&fa, k_mid<double, false>);
    else if (w.precision == BX_TF32X3) e = cudaFuncGetAttributes(&fa, k_mid<float, true>);
    else e = w.nes > 1 ? cudaFuncGetAttributes(&fa, k_mid32<true>) : cudaFuncGetAttributes(&fa, k_mid32<false>);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    *avail = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    return cudaSuccess;
}

cudaError_t launch_mid(const Work& w, int n, int Mmax, int nwmax, int Lmax, int want_grad, int want_mu,
                       cudaStream_t s) {
    const size_t smem = mid_dynamic_smem(w, Mmax, nwmax, Lmax);
    if (w.precision == BX_FP64) return launch_mid_t<double, false>(w, n, smem, want_grad, want_mu, s);
    if (w.precision == BX_TF32X3) return launch_mid_t<float, true>(w, n, smem, want_grad, want_mu, s);
    static size_t set32[2] = {0, 0};
    const int mes = w.nes > 1 ? 1 : 0;   // several energy slices of the Eq. 4 terms
    if (smem > set32[mes]) {
        const cudaError_t e = cudaFuncSetAttribute(mes ? k_mid32<true> : k_mid32<false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set32[mes] = smem;
    }
    if (mes) k_mid32<true><<<n, MID_THREADS, smem, s>>>(w, want_grad, want_mu);
    else k_mid32<false><<<n, MID_THREADS, smem, s>>>(w, want_grad, want_mu);
    return cudaGetLastError();
}

}  // namespace bx
