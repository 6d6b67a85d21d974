// bx_fwd_f32.cu -- Eq. 1 forward in FP32 on the CUDA cores (the mixed-precision path).
//
// Rate-first form: the Eq. 3 spectra are contracted directly,
//     lambda_h[m] = sum_i R[m,i] S_h[i],   S_h[i] = sum_k r_k c_{h,k} s_k[i]   (k_prep),
// and, for models with Eq. 4 terms, the response is also reduced over rows,
//     a_t[i] = sum_{m in tile t} R[m,i] Gg[m],
// from which k_mid forms every species' window marginal after pile-up.
// Unit = (row tile of TM output bins, item); 64 threads, each owning bins m0 + t and
// m0 + t + 64.  For every chunk of 32 true-energy columns of the tile's band the column
// parameters are staged in shared memory; each thread generates the response of its two
// bins with round-to-nearest FP32 arithmetic (bx_resp.cuh) and adds R S_h into
// Kahan-compensated accumulators at every term, so a row sum of ~10^3 terms keeps an error
// of a few roundings with no systematic sign.  Column sums go through a padded shared
// buffer (conflict-free in both directions) once per chunk.
#include <math.h>

#include "bx_internal.cuh"
#include "bx_resp.cuh"

namespace bx {

constexpr int F32_THREADS = TM / 2;
constexpr int FCH32 = 32;

__device__ __forceinline__ void kahan_fma(float& acc, float& cmp, float a, float b) {
    const float y = fmaf(a, b, -cmp);
    const float t = __fadd_rn(acc, y);
    cmp = __fsub_rn(__fsub_rn(t, acc), y);
    acc = t;
}

template <bool TAG, bool COLS>
__global__ void __launch_bounds__(F32_THREADS) k_fwd_f32(Work w) {
    const int tile = blockIdx.x, item = blockIdx.y, tid = threadIdx.x;
    const Toy& T = w.toys[w.toy_of[item]];
    if (tile >= T.n_tiles || w.status[item]) return;
    const int m0 = tile * TM, M = T.M;
    const int2 cr = w.tile_cols[(size_t)item * MAX_TILES + tile];
    const size_t cbase = (size_t)item * w.Npad;
    __shared__ float4 sC[FCH32];
    __shared__ ColG sG[FCH32];
    __shared__ float2 sS[FCH32];
    __shared__ float colbuf[COLS ? TM : 1][FCH32 + 1];
    __shared__ float colhalf[2][FCH32];

    const int ra = m0 + tid, rb = m0 + tid + F32_THREADS;
    const float mfa = (float)ra, mfb = (float)rb;
    const float gga = (COLS && ra < M) ? (float)T.Gg[ra] : 0.f;
    const float ggb = (COLS && rb < M) ? (float)T.Gg[rb] : 0.f;
    float sa = 0.f, csa = 0.f, ta = 0.f, cta = 0.f, sb = 0.f, csb = 0.f, tb = 0.f, ctb = 0.f;
    float* apart = static_cast<float*>(w.apart) + ((size_t)item * w.max_tiles + tile) * w.Npad;

    for (int c0 = cr.x; c0 < cr.y; c0 += FCH32) {
        if (tid < FCH32) {
            const bool in = c0 + tid < cr.y;
            sC[tid] = in ? w.colf[cbase + c0 + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
            sG[tid] = in ? w.colg[cbase + c0 + tid] : ColG{0.f, 0.f, 0.f, 0.f};
            const double2 S = in ? w.colS[cbase + c0 + tid] : make_double2(0.0, 0.0);
            sS[tid] = make_float2((float)S.x, (float)S.y);
        }
        __syncthreads();
        const int ncol = min(FCH32, cr.y - c0);
        for (int c = 0; c < ncol; ++c) {
            const float4 cf = sC[c];
            const ColG cg = sG[c];
            const float2 S = sS[c];
            const float Ra = resp_exact32(mfa, cf, cg), Rb = resp_exact32(mfb, cf, cg);
            kahan_fma(sa, csa, Ra, S.x);
            kahan_fma(sb, csb, Rb, S.x);
            if (TAG) {
                kahan_fma(ta, cta, Ra, S.y);
                kahan_fma(tb, ctb, Rb, S.y);
            }
            if (COLS) {
                colbuf[tid][c] = Ra * gga;
                colbuf[tid + F32_THREADS][c] = Rb * ggb;
            }
        }
        if (COLS) {
            __syncthreads();
            const int c = tid & 31, h = tid >> 5;
            float s = 0.f;
            for (int j = 0; j < F32_THREADS; ++j) s += colbuf[h * F32_THREADS + j][c];
            colhalf[h][c] = s;
            __syncthreads();
            if (tid < ncol) apart[c0 + tid] = colhalf[0][tid] + colhalf[1][tid];
        }
        __syncthreads();
    }
    double* lam = w.lam + (size_t)item * 2 * w.Mpad;
    if (ra < M) {
        lam[ra] = (double)sa - (double)csa;
        if (TAG) lam[w.Mpad + ra] = (double)ta - (double)cta;
    }
    if (rb < M) {
        lam[rb] = (double)sb - (double)csb;
        if (TAG) lam[w.Mpad + rb] = (double)tb - (double)ctb;
    }
}

cudaError_t launch_fwd_f32(const Work& w, int n, int max_tiles, int any_tag, int any_cols, cudaStream_t s) {
    dim3 grid(max_tiles, n);
    if (any_tag && any_cols) k_fwd_f32<true, true><<<grid, F32_THREADS, 0, s>>>(w);
    else if (any_tag) k_fwd_f32<true, false><<<grid, F32_THREADS, 0, s>>>(w);
    else if (any_cols) k_fwd_f32<false, true><<<grid, F32_THREADS, 0, s>>>(w);
    else k_fwd_f32<false, false><<<grid, F32_THREADS, 0, s>>>(w);
    return cudaGetLastError();
}

}  // namespace bx
