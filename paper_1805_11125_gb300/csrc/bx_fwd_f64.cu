// bx_fwd_f64.cu -- Eq. 1 forward in plain FP64 on the CUDA cores (the reference GPU form).
//
// Same rate-first reductions as the FP32 kernel (row sums lambda_h[m] = sum_i R[m,i] S_h[i]
// and per-tile column sums a_t,s[i] = sum_m R[m,i] Gg_s[m], one per energy slice s of the
// Eq. 4 terms), with the exact bin mass:
// unit = (row tile of TM output bins, item), thread = output bin.  For each chunk of
// FCH64 columns of the tile's band, phase 1 evaluates the Gaussian tail mass at the TM + 1
// bin edges of each column (one erfc per edge, shared by the two bins it bounds); phase 2
// forms R[m,i] = (Phi(z_{m+1}) - Phi(z_m)) / Phi(mu_i/sigma_i) from those tails without
// cancellation and accumulates the row sums; the column sums go through shared memory.  With a
// Gram-Charlier response every edge's tail takes the term -phi(z) C(z) of its CDF.
#include <math.h>

#include "bx_internal.cuh"

namespace bx {

constexpr int FCH64 = 16;   // columns per chunk

template <bool TAG, bool COLS>
__global__ void __launch_bounds__(TM) k_fwd_f64(Work w) {
    // 1D item-major grid (a y dimension would cap the batch at 65535 items)
    const int tile = blockIdx.x % w.max_tiles, item = blockIdx.x / w.max_tiles, tid = threadIdx.x;
    const Toy& T = w.toys[w.toy_of[item]];
    if (tile >= T.n_tiles || w.status[item]) return;
    const int m0 = tile * TM, M = T.M;
    const int NGRP = T.n_set > 1 ? T.n_set : 1;   // quenching groups: one column range each
    const size_t cbase = (size_t)item * w.Npad;
    const bool gc = T.gc1 != 0.0 || T.gc2 != 0.0;

    // tails, column-major so that thread = edge reads consecutive words
    __shared__ double sT[FCH64 * (TM + 1)];
    __shared__ unsigned char sF[FCH64 * (TM + 1)];   // 1: edge at or above the mean
    __shared__ double2 sS[FCH64];
    __shared__ double sNorm[FCH64];
    __shared__ double colbuf[COLS ? TM : 1][FCH64 + 1];   // R of the chunk's columns
    __shared__ double sGg[COLS ? MAX_ES : 1][TM];          // Gg_s of the tile's rows

    const int m = m0 + tid;
    const int NES = T.n_es;
    if (COLS)
        for (int q = 0; q < NES; ++q) sGg[q][tid] = m < M ? T.Gg[(size_t)q * M + m] : 0.0;
    double ls = 0.0, lt = 0.0;
    double* apart = static_cast<double*>(w.apart) + ((size_t)item * w.max_tiles + tile) * w.nes * w.Npad;

    for (int grp = 0; grp < NGRP; ++grp) {
    const int2 cr = tile_range(w, item, grp, tile);
    for (int c0 = cr.x; c0 < cr.y; c0 += FCH64) {
        for (int j = tid; j < FCH64 * (TM + 1); j += TM) {
            const int c = j / (TM + 1), e = j % (TM + 1), i = c0 + c;
            double t = 0.0;
            unsigned char f = 0;
            if (i < cr.y) {
                const Col64 cc = w.col64[cbase + i];
                const double z = ((double)(m0 + e) * T.w - cc.mu) / cc.sig;
                if (z >= 0.0) {
                    t = -0.5 * erfc(z * 0.70710678118654752440);   // -Q(z)
                    f = 1;
                } else {
                    t = 0.5 * erfc(-z * 0.70710678118654752440);   // Phi(z)
                }
                if (gc) t -= gc_cdf_term(T, z);   // the Gram-Charlier CDF: Phi(z) - phi(z) C(z)
            }
            sT[j] = t;
            sF[j] = f;
        }
        if (tid < FCH64) {
            const bool in = c0 + tid < cr.y;
            sS[tid] = in ? w.colS[cbase + c0 + tid] : make_double2(0.0, 0.0);
            sNorm[tid] = in ? w.col64[cbase + c0 + tid].norm : 0.0;
        }
        __syncthreads();
        const int ncol = min(FCH64, cr.y - c0);
        for (int c = 0; c < ncol; ++c) {
            const int ja = c * (TM + 1) + tid;
            // mass of [edge tid, edge tid+1]: same side -> difference of tails; straddling the
            // mean -> 1 - Q(z_b) - Phi(z_a)
            const double D = sT[ja + 1] - sT[ja] + ((!sF[ja] && sF[ja + 1]) ? 1.0 : 0.0);
            const double R = D * sNorm[c];
            ls = fma(R, sS[c].x, ls);
            if (TAG) lt = fma(R, sS[c].y, lt);
            if (COLS) colbuf[tid][c] = R;
        }
        if (COLS) {
            __syncthreads();
            // column c = tid / 8 summed by 8 threads over 16 rows each, once per energy slice
            const int c = tid >> 3, part = tid & 7;
            for (int q = 0; q < NES; ++q) {
                double s = 0.0;
                for (int j = 0; j < TM / 8; ++j) {
                    const int r = part * (TM / 8) + j;
                    s += colbuf[r][c] * sGg[q][r];
                }
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                if (part == 0 && c < ncol) apart[(size_t)q * w.Npad + c0 + c] = s;
            }
        }
        __syncthreads();
    }
    }
    if (m < M) {
        double* lam = w.lam + (size_t)item * 2 * w.Mpad;
        lam[m] = ls;
        if (TAG) lam[w.Mpad + m] = lt;
    }
}

cudaError_t launch_fwd_f64(const Work& w, int n, int max_tiles, int any_tag, int any_cols, cudaStream_t s) {
    const unsigned grid = (unsigned)n * (unsigned)w.max_tiles;   // decoded with w.max_tiles
    if (any_tag && any_cols) k_fwd_f64<true, true><<<grid, TM, 0, s>>>(w);
    else if (any_tag) k_fwd_f64<true, false><<<grid, TM, 0, s>>>(w);
    else if (any_cols) k_fwd_f64<false, true><<<grid, TM, 0, s>>>(w);
    else k_fwd_f64<false, false><<<grid, TM, 0, s>>>(w);
    return cudaGetLastError();
}

}  // namespace bx
