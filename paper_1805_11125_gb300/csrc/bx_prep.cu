// bx_prep.cu -- model set-up and the per-column stage of every evaluation.
//
// k_setup_toy (once per toy at model creation): FP32 copies of the shapes, the shapes
//   split into TF32 hi/lo tiles in the tensor-core operand layout, FP32 pile-up spectrum,
//   and the pile-up window marginal Gg[m] = sum_{m' in W, 0 <= m'-m < L} g[m'-m].
// k_prep (once per item): Eq. 1's Birks map and resolution on the true-energy grid in
//   FP64 (block-wide prefix sum), the column normalisation 1/Phi(mu/sigma), the FP32
//   parameters of the generated response and the band limits of every tile.
#include <float.h>
#include <limits.h>
#include <math.h>

#include "bx_internal.cuh"

namespace bx {

__global__ void k_setup_toy(Toy t, float* shapes32, float* S_tiles, float* g32, double* Gg) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int j = tid; j < t.K * t.N; j += nt) shapes32[j] = (float)t.shapes[j];
    // S tile of k-block kb: half h (0 = hi, 1 = lo), species row n, column c
    const int per_kb = 2 * US * KB;
    for (int j = tid; j < t.n_kb * per_kb; j += nt) {
        const int kb = j / per_kb, r = j % per_kb, h = r / (US * KB), e = r % (US * KB);
        const int n = e / KB, c = e % KB, i = kb * KB + c;
        const float s = (n < t.K && i < t.N) ? (float)t.shapes[(size_t)n * t.N + i] : 0.f;
        const float hi = tf32_rna(s);
        const float val = h == 0 ? hi : tf32_rna(s - hi);
        // K-major, no swizzle: 8x(4 x 4 B) core matrices; K step 256 B, 8-row step 128 B
        S_tiles[(size_t)kb * per_kb + h * US * KB + (c / 4) * (US * 4) + n * 4 + (c % 4)] = val;
    }
    for (int d = tid; d < t.L; d += nt) g32[d] = (float)t.g[d];
    for (int m = tid; m < t.M; m += nt) {
        double s = 0.0;
        const int lo = m > t.m_lo ? m : t.m_lo;
        const int hi = min(m + t.L - 1, t.M - 1);
        for (int mp = lo; mp <= hi; ++mp) s += t.g[mp - m];
        Gg[m] = s;
    }
}

cudaError_t launch_setup_toy(const Toy& t, float* shapes32, float* S_tiles, float* g32, double* Gg,
                             cudaStream_t s) {
    k_setup_toy<<<152, 256, 0, s>>>(t, shapes32, S_tiles, g32, Gg);
    return cudaGetLastError();
}

// Gaussian mass between standard scores a < b, from the tail away from the mean.
__device__ __forceinline__ double gauss_mass(double a, double b) {
    const double r = 0.70710678118654752440;
    if (a >= 0.0) return 0.5 * (erfc(a * r) - erfc(b * r));
    if (b <= 0.0) return 0.5 * (erfc(-b * r) - erfc(-a * r));
    return 1.0 - 0.5 * erfc(b * r) - 0.5 * erfc(-a * r);
}

// Block-wide exclusive scan of two doubles (256 threads).
__device__ void block_scan2(double& a, double& b, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double ta = __shfl_up_sync(0xffffffffu, ia, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += ta; ib += tb; }
    }
    if (lane == 31) { sh[wid] = ia; sh[8 + wid] = ib; }
    __syncthreads();
    if (wid == 0) {
        double wa = lane < 8 ? sh[lane] : 0.0, wb = lane < 8 ? sh[8 + lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            double ta = __shfl_up_sync(0xffffffffu, wa, o), tb = __shfl_up_sync(0xffffffffu, wb, o);
            if (lane >= o) { wa += ta; wb += tb; }
        }
        if (lane < 8) { sh[16 + lane] = wa - sh[lane]; sh[24 + lane] = wb - sh[8 + lane]; }
    }
    __syncthreads();
    a = sh[16 + wid] + ia - a;
    b = sh[24 + wid] + ib - b;
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_prep(Work w) {
    const int item = blockIdx.x, tid = threadIdx.x;
    if (w.skip && w.skip[item]) {   // uniform for the block: no barrier is skipped unevenly
        if (tid == 0) w.status[item] = STATUS_SKIPPED;
        return;
    }
    const Toy& T = w.toys[w.toy_of[item]];
    const int K = T.K, N = T.N, M = T.M;
    const double* th = w.theta + (size_t)item * w.tstride;
    __shared__ double sh[32];
    __shared__ int s_bad;
    __shared__ int s_tlo[MAX_TILES], s_thi[MAX_TILES], s_rlo[MAX_CB], s_rhi[MAX_CB];
    if (tid == 0) s_bad = 0;
    for (int j = tid; j < MAX_TILES; j += blockDim.x) { s_tlo[j] = INT_MAX; s_thi[j] = INT_MIN; }
    for (int j = tid; j < MAX_CB; j += blockDim.x) { s_rlo[j] = INT_MAX; s_rhi[j] = INT_MIN; }
    __syncthreads();
    if (tid < T.P && !isfinite(th[tid])) s_bad = 1;
    const double LY = th[K], a = th[K + 1], b = th[K + 2], c = th[K + 3], kB = th[K + 4];
    if (tid == 0 && (!(LY > 0.0) || (T.n_rad > 0 && !(th[K + 6] > 0.0)))) s_bad = 1;

    // a1: Q_i = sum_{j<i} x_j + x_i / 2, x_j = dE / (1 + kB S_j); dQ_i/dkB likewise.
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int i0 = tid * per, i1 = min(i0 + per, N);
    double sx = 0.0, sy = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double q = 1.0 + kB * T.stop_pow[i];
        sx += T.dE / q;
        sy += -T.dE * T.stop_pow[i] / (q * q);
    }
    double ex = sx, ey = sy;
    block_scan2(ex, ey, sh);
    const double w_ = T.w, band = w.band;
    Col64* col = w.col64 + (size_t)item * w.Npad;
    double2* cq = w.colq + (size_t)item * w.Npad;
    float4* cf = w.colf + (size_t)item * w.Npad;
    ColG* cg = w.colg + (size_t)item * w.Npad;
    double2* cs = w.colS + (size_t)item * w.Npad;
    double* aW = w.aW + (size_t)item * w.Npad;
    int bad = 0;
    unsigned long long inband = 0;
    for (int i = i0; i < i1; ++i) {
        const double S = T.stop_pow[i], q = 1.0 + kB * S;
        if (!(q > 0.0)) bad = 1;
        const double x = T.dE / q, y = -T.dE * S / (q * q);
        const double Q = ex + 0.5 * x, dQ = ey + 0.5 * y;
        ex += x;
        ey += y;
        const double mu = LY * Q;
        const double var = a * mu + b * mu * mu + c;
        if (!(var > 0.0)) bad = 1;
        const double sig = sqrt(fmax(var, 1e-300));
        const double z = mu / sig;
        const double Phi = 0.5 * erfc(-z * 0.70710678118654752440);
        const double phi = INV_SQRT_2PI * exp(-0.5 * z * z);
        const double norm = 1.0 / Phi;
        col[i] = Col64{mu, sig, norm, phi / Phi};
        cq[i] = make_double2(Q, dQ);
        const double u = mu / w_;
        const double jf = floor(u);
        const double hs = w_ / sig * S_EX2, cc = (0.5 - (u - jf)) * hs;
        const float hs_hi = (float)hs, c_hi = (float)cc;
        cf[i] = make_float4((float)jf, c_hi, hs_hi, (float)(hs - (double)hs_hi));
        const double kk = 0.38729833462074170 * hs;
        cg[i] = ColG{(float)(2.0 * 0.69314718055994531 * kk), (float)(2.0 * exp2(-kk * kk)),
                     (float)(cc - (double)c_hi), (float)(0.5 * (w_ / sig) * norm * INV_SQRT_2PI * GL_W_SCALE)};
        // rate-weighted shapes of the vetoed (or single) and tagged spectra (Eq. 3)
        double ssub = 0.0, stag = 0.0;
        for (int k = 0; k < K; ++k) {
            const double sk = T.shapes[(size_t)k * N + i] * th[k];
            const double t = T.tag ? T.tag[k] : 0.0;
            ssub += (T.tag ? 1.0 - t : 1.0) * sk;
            stag += t * sk;
        }
        cs[i] = make_double2(ssub, stag);
        // window mass of the column (Eq. 4 marginals)
        aW[i] = gauss_mass((T.m_lo * w_ - mu) / sig, (M * w_ - mu) / sig) * norm;
        // response band: rows whose bin lies within band * sigma of mu
        const double lo_e = fmin(fmax(mu - band * sig, -2.0 * w_), (M + 2.0) * w_);
        const double hi_e = fmin(fmax(mu + band * sig, -2.0 * w_), (M + 2.0) * w_);
        const int r0 = max(0, (int)floor(lo_e / w_));
        const int r1 = min(M, (int)floor(hi_e / w_) + 1);
        if (r0 < r1 && !bad) {
            inband += (unsigned long long)(r1 - r0);
            for (int t = r0 / TM; t <= (r1 - 1) / TM; ++t) {
                atomicMin(&s_tlo[t], i);
                atomicMax(&s_thi[t], i + 1);
            }
            atomicMin(&s_rlo[i / BCOLS], r0);
            atomicMax(&s_rhi[i / BCOLS], r1);
        }
    }
    for (int i = N + tid; i < w.Npad; i += blockDim.x) {
        col[i] = Col64{0.0, 1.0, 0.0, 0.0};
        cq[i] = make_double2(0.0, 0.0);
        cf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        cg[i] = ColG{0.f, 0.f, 0.f, 0.f};
        cs[i] = make_double2(0.0, 0.0);
        aW[i] = 0.0;
    }
    if (bad) s_bad = 1;
    if (w.count_units && inband) atomicAdd(w.units, inband);
    __syncthreads();
    for (int t = tid; t < MAX_TILES; t += blockDim.x)
        w.tile_cols[(size_t)item * MAX_TILES + t] = make_int2(s_tlo[t], s_thi[t]);
    for (int j = tid; j < MAX_CB; j += blockDim.x)
        w.cb_rows[(size_t)item * MAX_CB + j] = make_int2(s_rlo[j], s_rhi[j]);
    if (tid == 0) w.status[item] = s_bad ? (int)BX_EDOMAIN : 0;
}

cudaError_t launch_prep(const Work& w, int n, cudaStream_t s) {
    k_prep<<<n, 256, 0, s>>>(w);
    return cudaGetLastError();
}

}  // namespace bx
