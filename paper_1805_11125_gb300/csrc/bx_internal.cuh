// bx_internal.cuh -- device-side data layout and PTX helpers of the binned -lnL engine.
//
// One evaluation (an "item" = one toy at one parameter point) runs as
//   k_prep   per-column FP64 quantities of Eq. 1 (Birks map, mean, width, normalisation),
//            the rate-weighted shapes S_h[i] = sum_k r_k c_{h,k} s_k[i] of the Eq. 3
//            spectra, the window mass of every column, band limits, FP32 column parameters;
//   k_fwd_*  response generated on the fly (Eq. 1) and reduced both ways: row sums
//            lambda_h[m] = sum_i R[m,i] S_h[i] and, for the Eq. 4 terms, column sums
//            a[i] = sum_m R[m,i] Gg[m] (the tensor-core variant instead contracts with every
//            species shape, v[m][k] = sum_i R[m,i] s_k[i]);
//   k_mid    Eq. 2 pile-up, Eq. 4 marginals, -lnL (FP64, compensated), adjoint row weights;
//   k_bwd_*  adjoint of Eq. 1 per true-energy column: response parameters through the
//            chain rule to LY, a, b, c, kB, and the rates through sum_m R[m,i] wt_h[m];
//   k_gather final -lnL and gradient per item.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bx.h"

namespace bx {

constexpr int TM = 128;        // forward tile: output rows per unit (UMMA M)
constexpr int KB = 32;         // forward k-block: true-energy columns per step
constexpr int US = 16;         // UMMA N: species slots (K <= 16)
constexpr int KMAX = 16;
constexpr int PMAX = KMAX + 7;
constexpr int BCOLS = 128;     // backward unit: true-energy columns (one per thread)
constexpr int MAX_TILES = 64;  // rows per toy <= MAX_TILES * TM
constexpr int MAX_CB = 64;     // columns per toy <= MAX_CB * BCOLS
constexpr int MAX_RAD = 256;
constexpr int MAX_PSD = 256;
constexpr int MAX_L = 4096;
constexpr int NSL = 128;       // 2D model: slices per contraction (UMMA N), TFC spectra included

// Gauss-Legendre 3-point rule on [-1, 1]: nodes 0, +-sqrt(3/5), weights 8/9, 5/9.  The
// weights are applied as the exact integers 8 and 5 and the 1/9 is folded into the FP64
// column factor: the FP32 roundings of 8/9 and 5/9 are both upward and would scale every
// bin mass by 1 + 3e-8, a bias the likelihood cannot absorb.
constexpr float GL_NODE_HALF = 0.38729833462074170f;   // 0.5 * sqrt(3/5): node offset in bin units
constexpr float GL_W_MID = 8.0f;
constexpr float GL_W_OUT = 5.0f;
constexpr double GL_W_SCALE = 1.0 / 9.0;
// sqrt(0.5 * log2(e)): exp(-z^2 / 2) = 2^(-(z * S_EX2)^2)
constexpr double S_EX2 = 0.84932180028801904272;
constexpr double INV_SQRT_2PI = 0.39894228040143267794;

constexpr int GPN = 5 + KMAX;   // backward partials per column block: LY, a, b, c, kB, rates

enum : unsigned { ERR_TIMEOUT = 1u, ERR_TMEM = 2u };

// FP32 parameters of the outer Gauss-Legendre nodes of one column (see bx_resp.cuh).
// kk = sqrt(3/5)/2 * hs is the outer-node offset in the scaled variable.
struct __align__(16) ColG {
    float kap, Ck2, c_lo, A;   // 2 ln2 kk, 2 * 2^(-kk^2), low part of (1/2 - frac(mu/w)) hs, (h/2) norm / (9 sqrt(2 pi))
};

// Device description of one toy (dataset + its fixed model inputs).
constexpr int MAX_SETS = 4;   // groups of species-specific quenching, or radial shells of the response
constexpr int MAX_ES = 4;     // energy slices of the Eq. 4 radial and pulse-shape terms

struct Toy {
    int K, N, M, m_lo, nw, L, n_rad, n_psd, has_tag, nb, P;
    int n_tiles, n_cb, n_kb;
    // species-specific quenching: group c of species (Birks multiplier xi[c]) owns the response
    // columns [c Ncs, c Ncs + N); Next = (n_set - 1) Ncs + N columns in use (n_set = 1: Ncs =
    // Next = N, the plain model)
    int n_set, Ncs, Next;
    // energy slices of the Eq. 4 terms: slice s is the rows [es_lo[s], es_hi[s]) of the window,
    // with its own radial and pulse-shape histogram (n_es = 1: the whole window)
    int n_es;
    int es_lo[MAX_ES], es_hi[MAX_ES];
    int set_of[KMAX];
    double xi[MAX_SETS];
    // position-dependent response (n_shell > 0): the sets are radial shells instead of quenching
    // groups; shell c has the light yield LY lyf[c] (folded into its columns' Q) and carries every
    // species k with the weight shw[c][k], the species' fraction of events in the shell
    int n_shell;
    double lyf[MAX_SETS];
    double shw[MAX_SETS][KMAX];
    double dE, w, r_fid, r_iv, att_len;
    double gc1, gc2;          // Gram-Charlier response: skewness / 6 and excess kurtosis / 24 (0, 0: Gaussian)
    const double* shapes;     // [K][N]
    const float* shapes32;    // [K][N]
    const float* shapes32l;   // [K][N]: shapes - shapes32 (shapes32 + shapes32l is the FP64 shape to ~2^-48)
    const float* S_tiles;     // [n_kb][3][US*KB]: shapes split in three (split3), UMMA K-major
    const double* stop_pow;   // [N]
    const float2* stop32;     // [N]: the same as FP32 pairs hi + lo (nullptr: split on the fly)
    const double* tag;        // [K] or nullptr
    const double* g;          // [L]
    const float* g32;         // [L]
    const double* Gg;         // [n_es][M]: sum over the slice's window bins m' of g[m' - m] (0 <= m'-m < L)
    const float* Gg32;        // [n_es][M]: the same in FP32, stored after Gg
    const double* cnt;        // [nb] data, concatenated (vetoed, tagged, radial, PSD, 2D slices)
    const float2* cnt32;      // [nb] the same as FP32 pairs hi + lo
    const int* rad_class;     // [K]
    const double* psd;        // [K][n_psd]
    // 2D model (n_sl > 0): slices b = 0 vetoed, [1 tagged], then n_r2 radial and n_p2
    // pulse-shape slices of the vetoed events; counts are slice-major [n_sl][nw]
    int n_sl, n_r2, n_p2, b_r2;   // b_r2: first radial slice
    int joint2;                   // the 2D slices are the joint grid: slice b_r2 + rho n_p2 + j
    const float* ut;              // [N][NSL]: template modulation 1 + amp u[i][b] (1 for the TFC slices)
    const float* utl;             // [N][NSL]: (1 + amp u[i][b]) - ut[i][b], the low parts
    const double* U2;             // [K][NSL]: sum_i s_k[i] ut[i][b] (slice-set normalisation)
    const double* psd2;           // [K][n_p2]
    // template classes of the 2D model: within slice set s (0 vetoed, 1 tagged, 2 radial or the
    // joint grid, 3 pulse shape) species of one class share their slice probabilities q[b] (the
    // same radial class, the same pulse-shape row); cls_rep[s][c] is a species of class c
    int n_cls[4];
    int cls_of[4][KMAX], cls_rep[4][KMAX];
    const float* utmax;           // [NSL]: the largest ut[i][b] of each slice over the columns
};

// Weight of species k in the columns of set grp: a quenching group carries its own species
// (1, others 0), a radial shell every species with its fraction of events in the shell.
template <bool MULTI>
__host__ __device__ __forceinline__ double set_weight(const Toy& T, int k, int grp) {
    return !MULTI ? 1.0 : T.n_shell ? T.shw[grp][k] : (T.set_of[k] == grp ? 1.0 : 0.0);
}

// Per-column FP64 results of k_prep.
struct Col64 {
    double mu, sig, norm, mills;   // mean, width, 1/Phi(mu/sig), phi(mu/sig)/Phi(mu/sig)
};

// Workspace of a model: every array has `cap` item slots.
struct Work {
    int cap, Npad, Mpad, nbmax, pstride, n_items, max_tiles, max_cb;
    int nes;                  // energy slices of the Eq. 4 terms (the most of any toy, >= 1): the
                              // slice stride of aW, apart, rowW and coef
    int precision;
    int fwd_wpc;              // warps per CTA of the FP32 forward: 2 (0: default) or 1 (autotuner's choice)
    int gc;                   // some toy has a Gram-Charlier response (the FP32 kernels' GC instantiations)
    double band;
    unsigned long long watchdog_ns;
    const Toy* toys;
    const int* toy_of;        // [cap]
    const double* theta;      // [n][tstride]
    int tstride;
    Col64* col64;             // [cap][Npad]
    double2* colq;            // [cap][Npad]: Q_i, dQ_i/dkB
    float4* colf;             // [cap][Npad]: (floor(mu/w), c_hi, hs_hi, hs_lo): hs = w/sig*S_EX2, c = (1/2 - frac(mu/w)) hs
    ColG* colg;               // [cap][Npad]
    double2* colS;            // [cap][Npad]: S_vetoed[i], S_tagged[i] (FP64 model)
    float4* colS32;           // [cap][Npad]: A_i S_h[i] for the rate-first FP32 forward as double-float pairs
                              // (vetoed hi, tagged hi, vetoed lo, tagged lo)
    float* colAl;             // [cap][Npad]: A_i - colg[i].A, the low part of the column amplitude (the
                              // tensor-core forwards generate R = A_i x shape with it)
    double* aW;               // [cap][nes][Npad]: slice mass sum_{m in W_s} R[m,i] (closed form) times 1/Phi;
                              // as FP32 pairs (hi, lo) in the same bytes in the mixed-precision modes
    int2* colr;               // [cap][Npad]: band rows [r0, r1) of each column (empty: r0 >= r1)
    double* lam;              // [cap][2][Mpad]: lambda_h[m] (rate-first forward); FP32 pairs when lam_pairs
    int lam_pairs;            // rate-first mixed precision: the forward writes lam as FP32 pairs
    int multi_set;            // some toy has several quenching groups (selects the kernels that handle them)
    void* apart;              // [cap][max_tiles][H][nes][Npad]: column sums of R Gg_s per tile, FP64 (H = 1)
                              // or per half tile (one warp's 64 rows), FP32 (H = 2)
    int2* tile_cols;          // [cap][MAX_SETS][MAX_TILES]: column range of each forward tile, per
                              // quenching group (tile_range); only the toy's groups are written
    int2* cb_rows;            // [cap][MAX_CB]: row range of each backward column block
    void* v;                  // [2][cap][Mpad][US] float (TF32X3): species spectra v_k[m] as hi and lo planes
    void* rowW;               // [cap][2 + nes][Mpad] float or double: wt_sub, wt_tag, G_W of every slice
    double* coef;             // [cap][2 + nes][KMAX]: vetoed, tagged, then each slice's Eq. 4 coefficients
    double* gmid;             // [cap][PMAX]
    double* gpart;            // [cap][MAX_CB][GPN]
    double* nll;              // [cap]
    double* mu;               // [cap][nbmax]
    int* status;              // [cap]
    unsigned* err;            // sticky error word
    unsigned long long* units;   // in-band response entries evaluated (counted when count_units)
    int count_units;
    int shells;               // some toy has radial response shells (k_prep32's SHELL instantiations)
    const unsigned char* skip;   // [cap] or nullptr: items flagged 1 are not evaluated (-lnL = +inf)
    // 2D model buffers (UMMA K-major tiles of TF32 hi | lo halves, NSL slices x KB)
    float* coef2d;            // [cap][4][KMAX][NSL]: r_k dT/dr_k, dT/dr_k, r_k dT/ds_r coefficients, and the
                              // low part of the first (r_k dT/dr_k = plane 0 + plane 3 to ~2^-48)
    float* tr2d;              // [cap][tr_kb][3][NSL][KB]: rate-weighted templates (hi | mid | lo)
    unsigned* trmax2d;        // [cap][NSL]: largest |T_r[i,b]| of each slice over all columns (FP32 bits)
    float2* alpha2d;          // [cap][4][KMAX]: per slice set, a species' coefficient without its class
                              // probability (double-float): coef[k][b] = alpha[set(b)][k] q[b][class of k]
    float2* qcls2d;           // [cap][NSL][KMAX]: q[b][c], the slice probability of class c (double-float)
    float2* wcls2d;           // [cap][ncs2d][Npad]: class sums W[set, c][i] = sum_{k in c} alpha[set][k] s_k[i]
    int ncs2d;                // class-sum rows (the most over the toys of sum over sets of n_cls)
    float* y2d;               // [cap][row_kb][3][NSL][KB]: Y = R T_r over output rows (TF32 hi | lo, FP32 remainder)
    float* w2d;               // [cap][win_kb][2][NSL][KB]: 1 - n/mu over window rows
    float* wt2d;              // [cap][row_kb][2][NSL][KB]: pile-up-correlated weights over rows
    double* nll2d;            // [cap][MAX_TILES][2]: compensated -lnL partials per window tile
    double* geps2d;           // [cap][MAX_TILES]
    double* gpart2d;          // [cap][MAX_CB][GPN + 1]: response, rate and s_r partials
    int tr_kb, row_kb, win_kb, win_tiles, Lmax;
};

#ifdef __CUDACC__
// Gram-Charlier response (a Gaussian corrected by its skewness and excess kurtosis, the same
// mean and variance): phi(z) C(z) with C = gc1 He2 + gc2 He3 is what the CDF differs from Phi(z)
// by, F(z) = Phi(z) - phi(z) C(z); the density is phi(z) (1 + gc1 He3(z) + gc2 He4(z)).
__device__ __forceinline__ double gc_cdf_term(const Toy& T, double z) {
    const double z2 = z * z;
    return 0.39894228040143267794 * exp(-0.5 * z2) * (T.gc1 * (z2 - 1.0) + T.gc2 * z * (z2 - 3.0));
}
__device__ __forceinline__ double gc_density_factor(const Toy& T, double z) {
    const double z2 = z * z;
    return 1.0 + T.gc1 * z * (z2 - 3.0) + T.gc2 * (z2 * (z2 - 6.0) + 3.0);
}

// Column range [x, y) of forward tile t of an item's quenching group grp.
__device__ __forceinline__ int2 tile_range(const Work& w, int item, int grp, int t) {
    return w.tile_cols[((size_t)item * MAX_SETS + grp) * MAX_TILES + t];
}
#endif


constexpr int STATUS_SKIPPED = 1;   // item status of a skipped evaluation

// ------------------------------------------------------------------ launchers (host)
cudaError_t launch_setup_toy(const Toy& t, float* shapes32, float* shapes32l, float* S_tiles, float* g32, double* Gg,
                             cudaStream_t s);
cudaError_t launch_prep(const Work& w, int n, cudaStream_t s);
cudaError_t launch_fwd_f64(const Work& w, int n, int max_tiles, int any_tag, int any_cols, cudaStream_t s);
cudaError_t launch_fwd_tc(const Work& w, int n, int max_tiles, cudaStream_t s);
cudaError_t launch_fwd_f32(const Work& w, int n, int max_tiles, int any_tag, int any_cols, cudaStream_t s);
// Dynamic shared memory the assembly kernel needs per item for these sizes, and the most the
// device allows it (the opt-in limit less the kernel's static shared memory).
cudaError_t mid_smem_budget(const Work& w, int Mmax, int nwmax, int Lmax, size_t* need, size_t* avail);
cudaError_t launch_mid(const Work& w, int n, int Mmax, int nwmax, int Lmax, int want_grad, int want_mu,
                       cudaStream_t s);
cudaError_t launch_bwd(const Work& w, int n, int max_cb, cudaStream_t s);
cudaError_t launch_gather(const Work& w, int n, double* nll_out, double* grad_out, int want_grad, cudaStream_t s);
cudaError_t launch_eval2d(const Work& w, int n, int want_grad, int want_mu, int stage, cudaStream_t s);
cudaError_t launch_gather2d(const Work& w, int n, double* nll_out, double* grad_out, int want_grad, cudaStream_t s);
// several energy estimators: public item j = internal items j E .. j E + E - 1
constexpr int MAX_EST = 4;
cudaError_t launch_est_split(const double* theta, int tstride, int n, int E, const Toy* toys, const int* toy_of,
                             const unsigned char* skip, double* th_int, int Pi, unsigned char* skip_int, cudaStream_t s);
cudaError_t launch_est_join(const double* nll_int, const double* grad_int, int Pi, int n, int E, const Toy* toys,
                            const int* toy_of, double* nll, double* grad, int P, int want_grad, cudaStream_t s);
cudaError_t launch_umma_selftest(const float* A, const float* B, float* D, unsigned* err, cudaStream_t s);
cudaError_t launch_watchdog_selftest(unsigned* err, unsigned long long budget_ns, cudaStream_t s);

// ------------------------------------------------------------------ device helpers
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false when the time budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long budget_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > budget_ns) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared through the TMA unit; completes `bytes` on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ---- tcgen05 (5th-generation tensor core, accumulators in tensor memory)

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major operand:
// core matrices of 8 rows x 16 bytes; lbo = byte step between core matrices along K,
// sbo = byte step between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version 1 (tcgen05)
    return d;                 // base offset 0, relative LBO, swizzle none
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
// Three-part split x = hi + mid + lo of a row (or slice) of a k-block whose largest value is
// mx: hi = rint(x / 2^e) 2^e with 2^e = 2^(exponent of mx - 7), so |hi / 2^e| <= 256; mid and
// lo are the TF32 roundings of what remains (x - hi and x - hi - mid are exact in FP32).
// All hi of the row share the grid 2^e: a product of two hi parts is an integer below 2^16
// times 2^(e_A + e_B), and any sum of 32 of them is exact in FP32 whatever order or rounding
// the accumulator uses.  Rows whose largest value is below 2^-100 put everything into mid, lo.
struct Grid {
    float inv, scale;
};
__device__ __forceinline__ Grid hi_grid(float mx) {
    const int e = ((__float_as_int(mx) >> 23) & 0xFF) - 127 - 7;
    if (!(mx > 7.8886091e-31f)) return Grid{0.f, 0.f};   // 2^-100
    return Grid{__int_as_float((127 - e) << 23), __int_as_float((127 + e) << 23)};
}
// The same with a 7-bit hi (|hi / 2^e| <= 128): 2^e = 2^(exponent of mx - 6).
__device__ __forceinline__ Grid hi_grid7(float mx) {
    const int e = ((__float_as_int(mx) >> 23) & 0xFF) - 127 - 6;
    if (!(mx > 7.8886091e-31f)) return Grid{0.f, 0.f};   // 2^-100
    return Grid{__int_as_float((127 - e) << 23), __int_as_float((127 + e) << 23)};
}
__device__ __forceinline__ void split3(float x, Grid g, float& hi, float& mid, float& lo) {
    hi = rintf(x * g.inv) * g.scale;
    const float r = x - hi;
    mid = tf32_rna(r);
    lo = tf32_rna(r - mid);
}

__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor of kind::f16 with both operands BF16: D = F32, A = B = BF16 (the same
// type: kind::f16 takes one operand type for both), both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (+)= A B^T for one K = 16 step of BF16 operands (32 bytes of K, as one K = 8 step of TF32).
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Round to the nearest BF16 (as its 16-bit pattern); the three-part BF16 split of x on grid g:
// hi on the grid (exact in BF16: at most 8 significant bits), mid and lo the BF16 roundings of
// what remains (x - hi and x - hi - mid are exact in FP32).
__device__ __forceinline__ uint16_t bf16_rn(float x) {
    uint16_t r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ void split3_bf16(float x, Grid g, uint16_t& hi, uint16_t& mid, uint16_t& lo) {
    const float h = rintf(x * g.inv) * g.scale;
    const float r = x - h;
    hi = bf16_rn(h);
    mid = bf16_rn(r);
    lo = bf16_rn(r - bf16_val(mid));
}
// The four-part BF16 split (a second lo part, lo2, the BF16 rounding of what lo leaves; every
// remainder is exact in FP32): for an operand whose hi grid is coarse, so that mid and lo alone
// would leave ~2^-19 of the grid step.
__device__ __forceinline__ void split4_bf16(float x, Grid g, uint16_t& hi, uint16_t& mid, uint16_t& lo,
                                            uint16_t& lo2) {
    const float h = rintf(x * g.inv) * g.scale;
    const float r = x - h;
    hi = bf16_rn(h);
    mid = bf16_rn(r);
    const float r2 = r - bf16_val(mid);
    lo = bf16_rn(r2);
    lo2 = bf16_rn(r2 - bf16_val(lo));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 columns of 32-bit from tensor memory (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(r[j]);
}

// 32 lanes x 8 columns of 32-bit from tensor memory (warp w % 4 reads lanes 32 (w % 4) + 0..31).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* out) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) out[j] = __uint_as_float(r[j]);
}

// ---- compensated FP64 sums

struct Neu {
    double s, c;
};
__device__ __forceinline__ void neu_add(Neu& a, double x) {
    double t = a.s + x;
    a.c += fabs(a.s) >= fabs(x) ? (a.s - t) + x : (x - t) + a.s;
    a.s = t;
}
__device__ __forceinline__ Neu neu_merge(Neu a, Neu b) {
    neu_add(a, b.s);
    a.c += b.c;
    return a;
}

// log1p(x) - x in FP32 without cancellation for BC_XLO <= x <= BC_XHI.  With s = x / (2 + x)
// (|s| <= 1/3), log1p(x) = 2 atanh(s), so
//   log1p(x) - x = -x^2 / (2 + x) + 2 (s^3/3 + s^5/5 + ... + s^19/19) + O(2 s^21 / 21),
// the truncation below 1e-11; the two parts have the same sign for x < 0 and the series is
// under a tenth of the first part for x > 0, so the result carries FP32 relative error.
constexpr float BC_XLO = -0.5f, BC_XHI = 1.0f;
__device__ __forceinline__ float log1p_minus_x32(float x) {
    const float r = 1.0f / (2.0f + x);
    const float s = x * r, s2 = s * s;
    float p = 2.0f / 19.0f;
    p = fmaf(s2, p, 2.0f / 17.0f);
    p = fmaf(s2, p, 2.0f / 15.0f);
    p = fmaf(s2, p, 2.0f / 13.0f);
    p = fmaf(s2, p, 2.0f / 11.0f);
    p = fmaf(s2, p, 2.0f / 9.0f);
    p = fmaf(s2, p, 2.0f / 7.0f);
    p = fmaf(s2, p, 2.0f / 5.0f);
    p = fmaf(s2, p, 2.0f / 3.0f);
    return fmaf(s2 * s, p, -(x * x) * r);
}

// Baker-Cousins term (mu - n) + n ln(n/mu) (n > 0) and its weight 1 - n/mu in FP32 for
// x = (n - mu)/mu in [BC_XLO, BC_XHI] (every bin of a reasonable fit): written as
// n (log1p(x) - x) + (n - mu) x, a sum of two terms within a factor ~3 of the result, so the
// term carries an FP32 relative error with no systematic sign.  Other bins take the FP64
// form.  Returns false outside the range.
__device__ __forceinline__ bool bc_term32(double n, double mu, double& term, double& wb) {
    const float d = (float)(n - mu);
    const float x = d / (float)mu;
    if (!(x >= BC_XLO && x <= BC_XHI)) return false;
    term = (double)fmaf((float)n, log1p_minus_x32(x), d * x);
    wb = (double)(-x);
    return true;
}

// Shell integral of r^2 exp((r - r_iv)/lam): F and dF/dlam.
__device__ __forceinline__ void shell_F(double r, double r_iv, double lam, double& F, double& dF) {
    const double e = exp((r - r_iv) / lam);
    const double poly = lam * r * r - 2.0 * lam * lam * r + 2.0 * lam * lam * lam;
    F = e * poly;
    dF = e * (-(r - r_iv) / (lam * lam) * poly + (r * r - 4.0 * lam * r + 6.0 * lam * lam));
}

// SPECIES: the tensor-core forward's species-resolved spectra (else rate-first).  The
// rate-first FP32 variant is held to 64 registers so that two CTAs share an SM.

// Compensated FP32 sum (value s + c): TwoProduct of each term by FMA, TwoSum into the
// running sum, the same to merge partial sums across a warp.
struct Sum32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x), bb = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
        s = t;
    }
    // add a * (b + bl), bl a small correction of b
    __device__ __forceinline__ void add_prod(float a, float b, float bl) {
        const float p = __fmul_rn(a, b);
        c = fmaf(a, bl, __fadd_rn(c, fmaf(a, b, -p)));
        add(p);
    }
    __device__ __forceinline__ Sum32 warp_reduce() const {
        Sum32 r = *this;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, r.s, o), oc = __shfl_xor_sync(0xffffffffu, r.c, o);
            r.add(os);
            r.c = __fadd_rn(r.c, oc);
        }
        return r;
    }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

#endif  // __CUDACC__

}  // namespace bx
