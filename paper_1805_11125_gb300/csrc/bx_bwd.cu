// bx_bwd.cu -- adjoint of Eq. 1 and the gather of the final gradient.
//
// dNLL/dR[m,i] = sum_k s_k[i] (c0_k wt_sub[m] + c1_k wt_tag[m] + sum_s c_{2+s,k} G_W,s[m]) = W[m,i]
// (coefficients and row weights written by k_mid; one G_W per energy slice s of the Eq. 4
// terms, one slice unless the model has several).  Thread = true-energy column i; it
// recomputes the response of its band rows (nothing of the forward pass is stored) and
// forms the column sums
//     S0 = sum_m W R,   S1 = sum_m W norm dD/dmu_i,   S2 = sum_m W norm dD/dsigma_i,
//     rho_h = sum_m R wt_h[m]   (h = vetoed, tagged)
// with D the Gaussian bin mass and norm_i = 1 / Phi(mu_i / sigma_i); then
//     dNLL/dmu_i    = S1 - (phi/Phi)(x_i) / sigma_i * S0
//     dNLL/dsigma_i = S2 + (phi/Phi)(x_i) mu_i / sigma_i^2 * S0,      x_i = mu_i / sigma_i,
// the chain rule through mu_i = LY Q_i(kB), sigma_i^2 = a mu_i + b mu_i^2 + c gives the
// partial gradient of (LY, a, b, c, kB), and dNLL/dr_k gets
// sum_i s_k[i] (c_{vetoed,k} rho_vetoed[i] + c_{tagged,k} rho_tagged[i]).
//   k_bwd_f64: exact bin mass from erfc tails and exact derivatives -(phi(z_b) - phi(z_a))/sigma,
//              -(z_b phi(z_b) - z_a phi(z_a))/sigma, FP64 throughout (with a Gram-Charlier
//              response its CDF and density in place of Phi and phi).
//   k_bwd_f32: the same integrals by the forward pass's 3-point Gauss-Legendre rule
//              (integrands phi, t phi, (t^2 - 1) phi) in round-to-nearest FP32, down each
//              column by the row recurrence of bx_resp.cuh (adj_run), column sums
//              in FP32 per chunk of rows and FP64 across chunks, the chain rule in FP64; the
//              species sums and the rate products in FP32 (FP64 work is 64 FP32 operations'
//              worth of issue on GB300 and would otherwise dominate the column epilogue).
#include <limits.h>
#include <math.h>

#include "bx_internal.cuh"
#include "bx_resp.cuh"

namespace bx {

constexpr int RCH = 256;   // rows per staged chunk

__device__ __forceinline__ void chain_rule(const Col64& cc, const double2& q, const double* th, int K, double S0,
                                           double S1, double S2, double (&g)[GPN]) {
    const double LY = th[K], a = th[K + 1], b = th[K + 2];
    const double mu = cc.mu, sig = cc.sig;
    const double dmu = S1 - cc.mills / sig * S0;
    const double dsig = S2 + cc.mills * mu / (sig * sig) * S0;
    const double Gmu = dmu + dsig * (a + 2.0 * b * mu) / (2.0 * sig);
    g[0] = Gmu * q.x;                       // LY
    g[1] = dsig * mu / (2.0 * sig);         // a
    g[2] = dsig * mu * mu / (2.0 * sig);    // b
    g[3] = dsig / (2.0 * sig);              // c
    g[4] = Gmu * LY * q.y;                  // kB
}

// A column's place among the sets: column ie is grid point ig of set grp (a quenching group or a
// radial shell); species k contributes to it with the weight set_weight(T, k, grp).

// rate part: g[5 + k] = w_k s_k[i] (c_vetoed,k rho_vetoed + c_tagged,k rho_tagged) for the species
// of the column's set (grid point i, set grp, weight w_k)
template <bool MULTI>
__device__ __forceinline__ void rate_part(const Toy& T, int i, int grp, double rs, double rt, double (&g)[GPN]) {
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const double wk = k < T.K ? set_weight<MULTI>(T, k, grp) : 0.0;
        if (wk != 0.0) {
            const double t = T.tag ? T.tag[k] : 0.0;
            g[5 + k] = wk * T.shapes[(size_t)k * T.N + i] * ((T.tag ? 1.0 - t : 1.0) * rs + t * rt);
        } else {
            g[5 + k] = 0.0;
        }
    }
}

// FP32 shape of species k at grid point ig times its weight wk in the column's set (0 outside
// its quenching group: no load)
template <bool MULTI>
__device__ __forceinline__ float shape_w(const Toy& T, int k, int ig, float wk) {
    if (!MULTI) return T.shapes32[(size_t)k * T.N + ig];
    return wk != 0.f ? wk * T.shapes32[(size_t)k * T.N + ig] : 0.f;
}

__device__ __forceinline__ void block_sum_gp(double (&g)[GPN], double* red, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < GPN; ++j) {
        const double s = warp_sum(g[j]);
        if (lane == 0) red[wid * GPN + j] = s;
    }
    __syncthreads();
    if (threadIdx.x < GPN) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += red[q * GPN + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Species sums of the column's adjoint weights: vetoed, tagged, and one per energy slice q
// of the Eq. 4 terms (SA[q], 0 beyond the toy's slices).
template <bool MULTI>
__device__ __forceinline__ void column_weights(const Work& w, const Toy& T, int item, int i, int grp, bool ok,
                                               double& Ssub, double& Stag, double (&SA)[MAX_ES]) {
    const double* coef = w.coef + (size_t)item * (2 + w.nes) * KMAX;
    Ssub = Stag = 0.0;
    for (int q = 0; q < MAX_ES; ++q) SA[q] = 0.0;
    if (!ok) return;
    for (int k = 0; k < T.K; ++k) {
        const double wk = set_weight<MULTI>(T, k, grp);
        if (wk == 0.0) continue;
        const double s = wk * T.shapes[(size_t)k * T.N + i];
        Ssub += coef[k] * s;
        Stag += coef[KMAX + k] * s;
        for (int q = 0; q < T.n_es; ++q) SA[q] += coef[(2 + q) * KMAX + k] * s;
    }
}

template <bool MULTI>
__global__ void __launch_bounds__(BCOLS) k_bwd_f64(Work w) {
    // 1D item-major grid (a y dimension would cap the batch at 65535 items)
    const int cb = blockIdx.x % w.max_cb, item = blockIdx.x / w.max_cb, tid = threadIdx.x;
    const Toy& T = w.toys[w.toy_of[item]];
    if (cb >= T.n_cb) return;
    double* gp = w.gpart + ((size_t)item * MAX_CB + cb) * GPN;
    if (w.status[item]) {
        if (tid < GPN) gp[tid] = 0.0;
        return;
    }
    const int i = cb * BCOLS + tid;   // column (of quenching group grp, grid point ig)
    const int grp = MULTI ? i / T.Ncs : 0, ig = MULTI ? i - grp * T.Ncs : i;
    const bool ok = MULTI ? (i < T.Next && ig < T.N) : i < T.N;
    const int2 rr = w.cb_rows[(size_t)item * MAX_CB + cb];
    if (MULTI && rr.x >= rr.y) {   // no column of this block has support in its quenching group
        if (tid < GPN) gp[tid] = 0.0;
        return;
    }
    const int r0 = max(rr.x, max(0, T.m_lo - T.L + 1)), r1 = min(rr.y, T.M);
    double Ssub, Stag, SA[MAX_ES];
    column_weights<MULTI>(w, T, item, ig, grp, ok, Ssub, Stag, SA);
    const Col64 cc = ok ? w.col64[(size_t)item * w.Npad + i] : Col64{0.0, 1.0, 0.0, 0.0};
    const double* rw = static_cast<const double*>(w.rowW) + (size_t)item * (2 + w.nes) * w.Mpad;
    const int NES = T.n_es;
    __shared__ double sW[2 + MAX_ES][RCH];   // wt_sub, wt_tag, G_W of each energy slice
    __shared__ double red[GPN * (BCOLS / 32)];
    double S0 = 0.0, S1 = 0.0, S2 = 0.0, Rs = 0.0, Rt = 0.0;
    double ta = 0.0, pa = 0.0, zpa = 0.0;
    bool fa = false;
    const double inv_sig = 1.0 / cc.sig;
    const bool gc = T.gc1 != 0.0 || T.gc2 != 0.0;
    auto edge = [&](int e, double& t, double& p, double& zp, bool& f) {
        const double z = ((double)e * T.w - cc.mu) * inv_sig;
        f = z >= 0.0;
        t = f ? -0.5 * erfc(z * 0.70710678118654752440) : 0.5 * erfc(-z * 0.70710678118654752440);
        p = INV_SQRT_2PI * exp(-0.5 * z * z);
        if (gc) {   // Gram-Charlier: CDF Phi - phi C, density phi (1 + gc1 He3 + gc2 He4)
            t -= gc_cdf_term(T, z);
            p *= gc_density_factor(T, z);
        }
        zp = z * p;
    };
    if (ok && r0 < r1) edge(r0, ta, pa, zpa, fa);
    for (int c0 = r0; c0 < r1; c0 += RCH) {
        const int nr = min(RCH, r1 - c0);
        for (int j = tid; j < nr; j += BCOLS)
            for (int r = 0; r < 2 + NES; ++r) sW[r][j] = rw[(size_t)r * w.Mpad + c0 + j];
        __syncthreads();
        if (ok) {
            for (int j = 0; j < nr; ++j) {
                double tb, pb, zpb;
                bool fb;
                edge(c0 + j + 1, tb, pb, zpb, fb);
                double W = sW[0][j] * Ssub + sW[1][j] * Stag;
                for (int q = 0; q < NES; ++q) W += sW[2 + q][j] * SA[q];
                const double D = tb - ta + ((!fa && fb) ? 1.0 : 0.0);
                S0 += W * D;
                S1 -= W * (pb - pa);
                S2 -= W * (zpb - zpa);
                Rs += D * sW[0][j];
                Rt += D * sW[1][j];
                ta = tb; pa = pb; zpa = zpb; fa = fb;
            }
        }
        __syncthreads();
    }
    double g[GPN];
#pragma unroll
    for (int j = 0; j < GPN; ++j) g[j] = 0.0;
    if (ok) {
        const double* th = w.theta + (size_t)item * w.tstride;
        chain_rule(cc, w.colq[(size_t)item * w.Npad + i], th, T.K, cc.norm * S0, cc.norm * S1 * inv_sig,
                   cc.norm * S2 * inv_sig, g);
        rate_part<MULTI>(T, ig, grp, cc.norm * Rs, cc.norm * Rt, g);
    }
    block_sum_gp(g, red, gp);
}

// GC: the Gram-Charlier response, whose node sums are taken row by row (resp_adjoint32_gc): the
// row recurrence of the Gaussian does not carry the polynomial factor.
template <bool MULTI, bool MES, bool GC = false>
__global__ void __launch_bounds__(BCOLS, 7) k_bwd_f32(Work w) {
    // 1D item-major grid (a y dimension would cap the batch at 65535 items)
    const int cb = blockIdx.x % w.max_cb, item = blockIdx.x / w.max_cb, tid = threadIdx.x;
    const Toy& T = w.toys[w.toy_of[item]];
    if (cb >= T.n_cb) return;
    double* gp = w.gpart + ((size_t)item * MAX_CB + cb) * GPN;
    if (w.status[item]) {
        if (tid < GPN) gp[tid] = 0.0;
        return;
    }
    const int i = cb * BCOLS + tid;   // column (of quenching group grp, grid point ig)
    const int grp = MULTI ? i / T.Ncs : 0, ig = MULTI ? i - grp * T.Ncs : i;
    const bool ok = MULTI ? (i < T.Next && ig < T.N) : i < T.N;
    const int2 rr = w.cb_rows[(size_t)item * MAX_CB + cb];
    if (MULTI && rr.x >= rr.y) {   // no column of this block has support in its quenching group
        if (tid < GPN) gp[tid] = 0.0;
        return;
    }
    const int r0 = max(rr.x, max(0, T.m_lo - T.L + 1)), r1 = min(rr.y, T.M);
    // vetoed, tagged and the window (energy slice) coefficients per species; MES: several
    // energy slices of the Eq. 4 terms, each with its own row weight G_W,q and coefficients
    constexpr int NR = MES ? 2 + MAX_ES : 3;
    const int NES = MES ? T.n_es : 1;
    __shared__ float s_coef[NR][KMAX];
    __shared__ float s_c[2][KMAX];      // c_{vetoed,k}, c_{tagged,k}
    __shared__ float s_w[KMAX];         // MULTI: the species' weights in the block's set of columns
    __shared__ double red[GPN * (BCOLS / 32)];
    const double* coef = w.coef + (size_t)item * (2 + (MES ? w.nes : 1)) * KMAX;
    if (tid < (2 + NES) * KMAX) s_coef[tid / KMAX][tid % KMAX] = (float)coef[tid];
    // (a block's columns with support all lie in one set: Ncs is a multiple of BCOLS with several
    // sets, and with one set every column below N is set 0)
    if (MULTI && tid < KMAX) s_w[tid] = tid < T.K ? (float)set_weight<true>(T, tid, (cb * BCOLS) / T.Ncs) : 0.f;
    if (tid < KMAX) {
        const double t = (T.tag && tid < T.K) ? T.tag[tid] : 0.0;
        s_c[0][tid] = T.tag ? (float)(1.0 - t) : 1.f;
        s_c[1][tid] = (float)t;
    }
    __syncthreads();
    // dNLL/dR[m,i] = Ssub wt_sub[m] + Stag wt_tag[m] + sum_q SA_q G_W,q[m]: the species sums in FP32
    float Ssub = 0.f, Stag = 0.f, SA = 0.f;
    float SAq[MAX_ES] = {0.f, 0.f, 0.f, 0.f};   // MES: one sum per energy slice
    if constexpr (MES) {
        if (ok)
            for (int k0 = 0; k0 < T.K; k0 += 4) {
                float skv[4];
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const int k = k0 + q4;
                    skv[q4] = k < T.K ? shape_w<MULTI>(T, k, ig, s_w[k]) : 0.f;
                }
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const int k = k0 + q4;
                    if (k >= T.K) continue;
                    const float sk = skv[q4];
                    Ssub = fmaf(s_coef[0][k], sk, Ssub);
                    Stag = fmaf(s_coef[1][k], sk, Stag);
#pragma unroll
                    for (int q = 0; q < MAX_ES; ++q)
                        if (q < NES) SAq[q] = fmaf(s_coef[2 + q][k], sk, SAq[q]);
                }
            }
    } else {
        if (ok)   // four species' loads in flight at a time (a loop of load-then-use waits on each)
            for (int k0 = 0; k0 < T.K; k0 += 4) {
                float sk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = k0 + q;
                    sk[q] = k < T.K ? shape_w<MULTI>(T, k, ig, s_w[k]) : 0.f;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = k0 + q;
                    if (k < T.K) {
                        Ssub = fmaf(s_coef[0][k], sk[q], Ssub);
                        Stag = fmaf(s_coef[1][k], sk[q], Stag);
                        SA = fmaf(s_coef[2][k], sk[q], SA);
                    }
                }
            }
    }
    const float4 cf = ok ? w.colf[(size_t)item * w.Npad + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const ColG cg = ok ? w.colg[(size_t)item * w.Npad + i] : ColG{0.f, 0.f, 0.f, 0.f};
    const AdjCol ac = adj_col(cf, cg);
    const float* rw = static_cast<const float*>(w.rowW) + (size_t)item * (2 + (MES ? w.nes : 1)) * w.Mpad;
    // the warp's rows: the union of its 32 columns' bands, their weights staged 64 rows at a
    // time in the warp's own shared memory (the warps of the block never wait for each other)
    const int2 band = ok ? w.colr[(size_t)item * w.Npad + i] : make_int2(0, 0);
    const bool live = band.x < band.y;
    const int wr0 = max(r0, min(r1, __reduce_min_sync(0xffffffffu, live ? band.x : INT_MAX)));
    const int wr1 = min(r1, __reduce_max_sync(0xffffffffu, live ? band.y : 0));
    const int lane = tid & 31, wq = tid >> 5;
    // one energy slice: (wt_sub, wt_tag, G_W, -) packed per row (one 16-byte load; the row
    // weights do not depend on the column's set); several slices keep one row array per weight
    constexpr bool PACK = !MES;
    __shared__ float sW[BCOLS / 32][PACK ? 1 : NR][PACK ? 1 : 64];
    __shared__ float4 sW4[BCOLS / 32][PACK ? 64 : 1];
    double S0 = 0.0, S1 = 0.0, S2 = 0.0, Rs = 0.0, Rt = 0.0;
    const float gc3 = GC ? (float)T.gc1 : 0.f, gc4 = GC ? (float)T.gc2 : 0.f;
    for (int c0 = wr0; c0 < wr1; c0 += RCH) {
        const int c1 = min(wr1, c0 + RCH);
        AdjSums bs;
        float q0 = 0.f, q1 = 0.f, q2 = 0.f, qs = 0.f, qt = 0.f;   // GC: the chunk's node sums
        for (int s0 = c0; s0 < c1; s0 += 64) {
            const int ns = min(64, c1 - s0);
            for (int j = lane; j < ns; j += 32) {
                if constexpr (PACK) {
                    sW4[wq][j] = make_float4(rw[s0 + j], rw[(size_t)w.Mpad + s0 + j], rw[(size_t)2 * w.Mpad + s0 + j], 0.f);
                } else {
                    sW[wq][0][j] = rw[s0 + j];
                    sW[wq][1][j] = rw[(size_t)w.Mpad + s0 + j];
                    for (int q = 0; q < NES; ++q) sW[wq][2 + q][j] = rw[(size_t)(2 + q) * w.Mpad + s0 + j];
                }
            }
            __syncwarp();
            if (GC && ok) {   // row by row
                for (int j = 0; j < ns; ++j) {
                    float ws, wt, W;
                    if constexpr (MES) {
                        ws = sW[wq][0][j];
                        wt = sW[wq][1][j];
                        float a = 0.f;
#pragma unroll
                        for (int q = 0; q < MAX_ES; ++q)
                            if (q < NES) a = fmaf(sW[wq][2 + q][j], SAq[q], a);
                        W = fmaf(ws, Ssub, fmaf(wt, Stag, a));
                    } else if constexpr (PACK) {
                        const float4 rr = sW4[wq][j];
                        ws = rr.x;
                        wt = rr.y;
                        W = fmaf(ws, Ssub, fmaf(wt, Stag, rr.z * SA));
                    } else {
                        ws = sW[wq][0][j];
                        wt = sW[wq][1][j];
                        W = fmaf(ws, Ssub, fmaf(wt, Stag, sW[wq][2][j] * SA));
                    }
                    float P0, P1, P2;
                    resp_adjoint32_gc((float)(s0 + j), cf, cg, gc3, gc4, P0, P1, P2);
                    q0 = fmaf(W, P0, q0);
                    q1 = fmaf(W, P1, q1);
                    q2 = fmaf(W, P2, q2);
                    qs = fmaf(ws, P0, qs);
                    qt = fmaf(wt, P0, qt);
                }
            } else if (ok) {
                for (int j = 0; j < ns; j += ADJ_RUN) {
                    if constexpr (MES) {
                        auto wts = [&](int k, float& ws, float& wt, float& W) {
                            ws = sW[wq][0][j + k];
                            wt = sW[wq][1][j + k];
                            float a = 0.f;
#pragma unroll
                            for (int q = 0; q < MAX_ES; ++q)
                                if (q < NES) a = fmaf(sW[wq][2 + q][j + k], SAq[q], a);
                            W = fmaf(ws, Ssub, fmaf(wt, Stag, a));
                        };
                        adj_run((float)(s0 + j), min(ADJ_RUN, ns - j), cf, cg, ac, wts, bs);
                    } else if constexpr (PACK) {
                        auto wts = [&](int k, float& ws, float& wt, float& W) {
                            const float4 r = sW4[wq][j + k];
                            ws = r.x;
                            wt = r.y;
                            W = fmaf(ws, Ssub, fmaf(wt, Stag, r.z * SA));
                        };
                        adj_run((float)(s0 + j), min(ADJ_RUN, ns - j), cf, cg, ac, wts, bs);
                    } else {
                        auto wts = [&](int k, float& ws, float& wt, float& W) {
                            ws = sW[wq][0][j + k];
                            wt = sW[wq][1][j + k];
                            W = fmaf(ws, Ssub, fmaf(wt, Stag, sW[wq][2][j + k] * SA));
                        };
                        adj_run((float)(s0 + j), min(ADJ_RUN, ns - j), cf, cg, ac, wts, bs);
                    }
                }
            }
            __syncwarp();
        }
        float p0, p1, p2, ps, pt;
        if (GC) {
            p0 = q0;
            p1 = q1;
            p2 = q2;
            ps = qs;
            pt = qt;
        } else {
            bs.node(cg.Ck2, ac.kk, p0, p1, p2, ps, pt);
        }
        S0 += p0;
        S1 += p1;
        S2 += p2;
        Rs += ps;
        Rt += pt;
    }
    // chain rule through mu_i = LY Q_i(kB), sigma_i^2 = a mu_i + b mu_i^2 + c in FP64
    double g5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    float rho_s = 0.f, rho_t = 0.f;
    if (ok) {
        const Col64 cc = w.col64[(size_t)item * w.Npad + i];
        const double2 q = w.colq[(size_t)item * w.Npad + i];
        const double* th = w.theta + (size_t)item * w.tstride;
        const double LY = th[T.K], a = th[T.K + 1], b = th[T.K + 2];
        const double isig = 1.0 / cc.sig;
        const double A = (0.5 * INV_SQRT_2PI * GL_W_SCALE) * T.w * isig * cc.norm;   // R = A * P0
        // P1, P2 carry the node positions in units of z * S_EX2
        const double s0 = A * S0;
        const double s1 = A * isig * (S1 * (1.0 / S_EX2));
        const double s2 = A * isig * (S2 * (1.0 / (S_EX2 * S_EX2)) - S0);
        const double dmu = s1 - cc.mills * isig * s0;
        const double dsig = s2 + cc.mills * cc.mu * isig * isig * s0;
        const double D = 0.5 * isig * dsig;
        const double Gmu = dmu + D * (a + 2.0 * b * cc.mu);
        g5[0] = Gmu * q.x;               // LY
        g5[1] = D * cc.mu;               // a
        g5[2] = D * cc.mu * cc.mu;       // b
        g5[3] = D;                       // c
        g5[4] = Gmu * LY * q.y;          // kB
        rho_s = (float)(A * Rs);
        rho_t = (float)(A * Rt);
    }
    const int wid = wq;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const double v = warp_sum(g5[j]);
        if (lane == 0) red[wid * GPN + j] = v;
    }
    // rate part sum_i s_k[i] (c_vetoed,k rho_vetoed[i] + c_tagged,k rho_tagged[i]) in FP32 within
    // the warp (32 columns), FP64 from there on; the tensor-core path gets it from k_mid
    const bool rates = w.precision != BX_TF32X3;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < T.K && rates) {
            const float sk = ok ? shape_w<MULTI>(T, k, ig, s_w[k]) : 0.f;
            const float v = warp_sum(sk * fmaf(s_c[0][k], rho_s, s_c[1][k] * rho_t));
            if (lane == 0) red[wid * GPN + 5 + k] = (double)v;
        } else if (lane == 0) {
            red[wid * GPN + 5 + k] = 0.0;
        }
    }
    __syncthreads();
    if (tid < GPN) {
        double v = 0.0;
        for (int q = 0; q < BCOLS / 32; ++q) v += red[q * GPN + tid];
        gp[tid] = v;
    }
}

cudaError_t launch_bwd(const Work& w, int n, int max_cb, cudaStream_t s) {
    const unsigned grid = (unsigned)n * (unsigned)w.max_cb;   // decoded with w.max_cb
    if (w.precision == BX_FP64) {
        if (w.multi_set) k_bwd_f64<true><<<grid, BCOLS, 0, s>>>(w);
        else k_bwd_f64<false><<<grid, BCOLS, 0, s>>>(w);
    } else {
        const bool mes = w.nes > 1;   // several energy slices of the Eq. 4 terms
        if (w.gc) {   // the Gram-Charlier response (one quenching group)
            if (w.multi_set && mes) k_bwd_f32<true, true, true><<<grid, BCOLS, 0, s>>>(w);
            else if (w.multi_set) k_bwd_f32<true, false, true><<<grid, BCOLS, 0, s>>>(w);
            else if (mes) k_bwd_f32<false, true, true><<<grid, BCOLS, 0, s>>>(w);
            else k_bwd_f32<false, false, true><<<grid, BCOLS, 0, s>>>(w);
        } else if (w.multi_set && mes) k_bwd_f32<true, true><<<grid, BCOLS, 0, s>>>(w);
        else if (w.multi_set) k_bwd_f32<true, false><<<grid, BCOLS, 0, s>>>(w);
        else if (mes) k_bwd_f32<false, true><<<grid, BCOLS, 0, s>>>(w);
        else k_bwd_f32<false, false><<<grid, BCOLS, 0, s>>>(w);
    }
    return cudaGetLastError();
}

// Final -lnL and gradient of each item (rows of stride pstride; unused slots zeroed).
__global__ void k_gather(Work w, int n, double* nll_out, double* grad_out, int want_grad) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= n) return;
    const Toy& T = w.toys[w.toy_of[item]];
    const int st = w.status[item];
    nll_out[item] = st ? INFINITY : w.nll[item];
    if (!want_grad) return;
    const double* gm = w.gmid + (size_t)item * PMAX;
    const double* gp = w.gpart + (size_t)item * MAX_CB * GPN;
    double* go = grad_out + (size_t)item * w.pstride;
    for (int j = 0; j < w.pstride; ++j) {
        double g = 0.0;
        if (!st && j < T.P) {
            g = gm[j];
            int slot = -1;
            if (j < T.K) slot = 5 + j;
            else if (j < T.K + 5) slot = j - T.K;
            if (slot >= 0)
                for (int cb = 0; cb < T.n_cb; ++cb) g += gp[cb * GPN + slot];
        }
        go[j] = g;
    }
}

cudaError_t launch_gather(const Work& w, int n, double* nll_out, double* grad_out, int want_grad, cudaStream_t s) {
    k_gather<<<(n + 127) / 128, 128, 0, s>>>(w, n, nll_out, grad_out, want_grad);
    return cudaGetLastError();
}

}  // namespace bx
