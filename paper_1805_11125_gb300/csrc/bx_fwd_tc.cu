// bx_fwd_tc.cu -- Eq. 1 forward on the 5th-generation tensor cores (tcgen05, sm_103a), the
// species-resolved form v_k[m] = sum_i R[m,i] s_k[i] (BX_TF32X3).
//
// Unit = (row tile of TM = 128 output bins, item); 512 threads, thread = (row r, quarter h of
// a k-block's KB = 32 true-energy columns).  For every k-block of the tile's band:
//   * one thread starts a bulk copy of the k-block's species tile, split in three at model
//     creation (split3: an 8-bit hi on a grid shared by the species row of the k-block, then
//     TF32 mid and lo) and pre-arranged in the UMMA K-major layout;
//   * the CUDA cores generate the 128 x 32 response tile with the bias-free FP32 generator of
//     bx_resp.cuh and split it in three on a grid shared by each row;
//   * one thread issues the five cross products (smallest first) into a fresh TMEM region S
//     and hi * hi into a fresh region E (M = 128, N = 16, K = 8 per instruction).  Every
//     hi * hi product is an integer below 2^16 on one power-of-two grid, so E is exact
//     whatever the accumulator's rounding; S holds values 2^-8 of E or less, so the FP32
//     accumulator's truncation toward zero acts only on those.
// Two stages alternate: the generation of k-block j overlaps the MMAs of j - 1, and the
// regions of k-block j are drained into Kahan-compensated FP32 sums when j + 2 starts.
// Every wait is bounded by the watchdog budget; on expiry the CTA records ERR_TIMEOUT,
// waits (bounded, at least 2 s) for its own bulk copies and MMAs, frees its tensor memory
// and returns.
#include <math.h>

#include "bx_internal.cuh"
#include "bx_resp.cuh"

namespace bx {

constexpr int TC_THREADS = 512;
constexpr int A_FLOATS1 = TM * KB;          // one part of a response tile
constexpr int S3_FLOATS = 3 * US * KB;      // species tile hi | mid | lo
constexpr uint32_t S3_BYTES = S3_FLOATS * 4;
constexpr uint32_t TMEM_COLS = 4 * US;      // two stages x (S, E) x 16 species
constexpr unsigned long long TC_CLEANUP_NS = 2000000000ull;

struct __align__(128) SmemTC {
    float A[2][3][A_FLOATS1];   // response tiles, hi | mid | lo
    float B[2][S3_FLOATS];      // species tiles
    float4 colf[KB];
    ColG colg[KB];
    float colal[KB];
    float rowmax[4][TM];
    uint64_t mma_bar[2];
    uint64_t b_bar[2];
    uint32_t tmem_base;
    int abort;
    int committed;
};

// A (128 x 32, K-major): element (r, c) at (c / 4) * 512 + r * 4 + c % 4
__device__ __forceinline__ int tc_a_off(int r, int c) { return (c >> 2) * (TM * 4) + r * 4 + (c & 3); }

// One k-block: region S (fresh) <- hi_A lo_B, lo_A hi_B, mid_A mid_B, hi_A mid_B, mid_A hi_B;
// region E (fresh) <- hi_A hi_B.  A3: parts at stride A_FLOATS1; B3: parts at stride US * KB.
__device__ __forceinline__ void mma_kblock3_species(uint32_t dS, uint32_t dE, const float* A3, const float* B3) {
    constexpr uint32_t idesc = umma_idesc_tf32(TM, US);
    const uint32_t a[3] = {smem_u32(A3), smem_u32(A3 + A_FLOATS1), smem_u32(A3 + 2 * A_FLOATS1)};
    const uint32_t b[3] = {smem_u32(B3), smem_u32(B3 + US * KB), smem_u32(B3 + 2 * US * KB)};
    constexpr int pa[5] = {0, 2, 1, 0, 1}, pb[5] = {2, 0, 1, 1, 0};
    uint32_t acc = 0u;
#pragma unroll
    for (int p = 0; p < 5; ++p)
#pragma unroll
        for (int q = 0; q < KB / 8; ++q) {
            // one K = 8 step spans two core-matrix columns
            umma_tf32(dS, umma_desc(a[pa[p]] + q * 2 * (TM * 16), TM * 16, 128),
                      umma_desc(b[pb[p]] + q * 2 * (US * 16), US * 16, 128), idesc, acc);
            acc = 1u;
        }
#pragma unroll
    for (int q = 0; q < KB / 8; ++q)
        umma_tf32(dE, umma_desc(a[0] + q * 2 * (TM * 16), TM * 16, 128), umma_desc(b[0] + q * 2 * (US * 16), US * 16, 128),
                  idesc, q > 0 ? 1u : 0u);
}

// Split this thread's 8 values of row r (columns 8 h .. 8 h + 7) on the row's grid and store
// the three parts; the row maximum is combined over the four quarters through shared memory
// (the caller has stored rowmax[h][r] and synchronised).
__device__ __forceinline__ void store_split3(float* A3, const float (&x)[8], int r, int h, Grid g) {
#pragma unroll
    for (int c4 = 0; c4 < 2; ++c4) {
        float4 vh, vm, vl;
        split3(x[4 * c4 + 0], g, vh.x, vm.x, vl.x);
        split3(x[4 * c4 + 1], g, vh.y, vm.y, vl.y);
        split3(x[4 * c4 + 2], g, vh.z, vm.z, vl.z);
        split3(x[4 * c4 + 3], g, vh.w, vm.w, vl.w);
        const int o = tc_a_off(r, 8 * h + 4 * c4);
        *reinterpret_cast<float4*>(A3 + o) = vh;
        *reinterpret_cast<float4*>(A3 + A_FLOATS1 + o) = vm;
        *reinterpret_cast<float4*>(A3 + 2 * A_FLOATS1 + o) = vl;
    }
}

// Kahan-compensated drain of both regions of stage s into the 8 species sums of this thread:
// warps 0-7, lanes 32 (warp % 4) + lane, species 8 (warp / 4) .. + 7.
__device__ __forceinline__ void drain_species(uint32_t tbase, int s, float (&acc)[8], float (&cmp)[8]) {
    const int warp = threadIdx.x >> 5;
    const uint32_t lanes = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 8);
    float vS[8], vE[8];
    tmem_ld8(lanes + (uint32_t)(2 * s * US), vS);
    tmem_ld8(lanes + (uint32_t)((2 * s + 1) * US), vE);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float y = __fsub_rn(__fadd_rn(vE[q], vS[q]), cmp[q]);
        const float t = __fadd_rn(acc[q], y);
        cmp[q] = __fsub_rn(__fsub_rn(t, acc[q]), y);
        acc[q] = t;
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_fwd_tc(Work w) {
    extern __shared__ unsigned char smem_raw[];
    SmemTC& sm = *reinterpret_cast<SmemTC*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    // 1D item-major grid (a y dimension would cap the batch at 65535 items)
    const int tile = blockIdx.x % w.max_tiles, item = blockIdx.x / w.max_tiles, tid = threadIdx.x;
    const Toy& T = w.toys[w.toy_of[item]];
    if (tile >= T.n_tiles || w.status[item]) return;
    const int m0 = tile * TM, r = tid & (TM - 1), h = tid >> 7, warp = tid >> 5;
    const int2 cr = tile_range(w, item, 0, tile);   // one quenching group
    const int kb0 = cr.x < cr.y ? cr.x / KB : 0;
    const int nblk = cr.x < cr.y ? (cr.y - 1) / KB + 1 - kb0 : 0;
    const float4* colf = w.colf + (size_t)item * w.Npad;
    const ColG* colg = w.colg + (size_t)item * w.Npad;
    const float* colal = w.colAl + (size_t)item * w.Npad;
    const float* Sg = T.S_tiles + (size_t)kb0 * S3_FLOATS;
    float acc[8], cmp[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = cmp[q] = 0.f;
    bool ok = true;
    if (nblk > 0) {
        if (tid == 0) {
            mbar_init(&sm.mma_bar[0], 1);
            mbar_init(&sm.mma_bar[1], 1);
            mbar_init(&sm.b_bar[0], 1);
            mbar_init(&sm.b_bar[1], 1);
            sm.abort = 0;
            fence_mbar_init();
        }
        if (warp == 0) {
            tmem_alloc(&sm.tmem_base, TMEM_COLS);
            tmem_relinquish();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t tbase = sm.tmem_base;
        int issued = 0, waited = 0, committed = 0;   // thread 0 bookkeeping
        const float mf = (float)(m0 + r);
        const bool row_ok = m0 + r < T.M;
        for (int it = 0; it < nblk; ++it) {
            const int s = it & 1;
            // k-block it - 2 used stage s: its MMAs must be done before A, B and TMEM of s are reused
            if (it >= 2 && !mbar_wait(&sm.mma_bar[s], ((it - 2) >> 1) & 1, w.watchdog_ns)) atomicOr(&sm.abort, 1);
            if (tid < KB) {
                const int i = (kb0 + it) * KB + tid;
                const bool in = i < T.N;
                sm.colf[tid] = in ? colf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                sm.colg[tid] = in ? colg[i] : ColG{0.f, 0.f, 0.f, 0.f};
                sm.colal[tid] = in ? colal[i] : 0.f;
            }
            tc_fence_after();
            __syncthreads();
            if (sm.abort) break;
            if (it >= 2 && warp < 8) drain_species(tbase, s, acc, cmp);
            if (tid == 0) {
                mbar_arrive_expect_tx(&sm.b_bar[s], S3_BYTES);
                bulk_g2s(sm.B[s], Sg + (size_t)it * S3_FLOATS, S3_BYTES, &sm.b_bar[s]);
                ++issued;
            }
            const int ibase = (kb0 + it) * KB;
            float x[8];
            float mx = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = 8 * h + q;
                x[q] = (row_ok && ibase + c < T.N) ? resp_amp32(mf, sm.colf[c], sm.colg[c], sm.colal[c]) : 0.f;
                mx = fmaxf(mx, x[q]);
            }
            sm.rowmax[h][r] = mx;
            __syncthreads();
            const Grid g = hi_grid(fmaxf(fmaxf(sm.rowmax[0][r], sm.rowmax[1][r]), fmaxf(sm.rowmax[2][r], sm.rowmax[3][r])));
            store_split3(sm.A[s][0], x, r, h, g);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                if (!mbar_wait(&sm.b_bar[s], (it >> 1) & 1, w.watchdog_ns)) {
                    atomicOr(&sm.abort, 1);
                } else {
                    ++waited;
                    mma_kblock3_species(tbase + (uint32_t)(2 * s * US), tbase + (uint32_t)((2 * s + 1) * US), sm.A[s][0],
                                        sm.B[s]);
                    umma_commit(&sm.mma_bar[s]);
                    ++committed;
                }
            }
        }
        // Drain: every bulk copy and MMA of this CTA must have landed before the CTA frees its
        // tensor memory or exits (bounded by the larger of the watchdog and TC_CLEANUP_NS).
        if (tid == 0) {
            bool drained = true;
            for (int j = waited; j < issued; ++j) drained &= mbar_wait(&sm.b_bar[j & 1], (j >> 1) & 1, TC_CLEANUP_NS);
            if (!drained) atomicOr(&sm.abort, 1);
            sm.committed = committed;
        }
        __syncthreads();
        const int nc = sm.committed;
        const unsigned long long budget = w.watchdog_ns > TC_CLEANUP_NS ? w.watchdog_ns : TC_CLEANUP_NS;
        bool done = true;
        // the last two k-blocks (one per stage) are still to be waited for and drained
        for (int j = (nc >= 2 ? nc - 2 : 0); j < nc; ++j) done &= mbar_wait(&sm.mma_bar[j & 1], (j >> 1) & 1, budget);
        tc_fence_after();
        ok = !sm.abort && done && nc == nblk;
        if (ok && warp < 8)
            for (int j = (nc >= 2 ? nc - 2 : 0); j < nc; ++j) drain_species(tbase, j & 1, acc, cmp);
        if (!ok && tid == 0) atomicOr(w.err, ERR_TIMEOUT);
        tc_fence_before();
        __syncthreads();
        if (warp == 0) tmem_dealloc(tbase, TMEM_COLS);
    }
    // v rows: warps 0-7, row 32 (warp % 4) + lane of the tile, species 8 (warp / 4) .. + 7
    if (warp < 8) {
        const int row = m0 + (warp & 3) * 32 + (tid & 31);
        if (row < T.M) {
            // the Kahan sum acc - cmp as a normalised pair: hi plane, then the lo plane cap x Mpad x US later
            float* vrow = static_cast<float*>(w.v) + ((size_t)item * w.Mpad + row) * US + (warp >> 2) * 8;
            float* vlow = vrow + (size_t)w.cap * w.Mpad * US;
            float o[8], l[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                o[q] = ok ? __fsub_rn(acc[q], cmp[q]) : 0.f;
                l[q] = ok ? __fsub_rn(__fsub_rn(acc[q], o[q]), cmp[q]) : 0.f;
            }
            *reinterpret_cast<float4*>(vrow) = make_float4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<float4*>(vrow + 4) = make_float4(o[4], o[5], o[6], o[7]);
            *reinterpret_cast<float4*>(vlow) = make_float4(l[0], l[1], l[2], l[3]);
            *reinterpret_cast<float4*>(vlow + 4) = make_float4(l[4], l[5], l[6], l[7]);
        }
    }
}

cudaError_t launch_fwd_tc(const Work& w, int n, int max_tiles, cudaStream_t s) {
    const int smem = (int)sizeof(SmemTC) + 128;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const unsigned grid = (unsigned)n * (unsigned)w.max_tiles;   // decoded with w.max_tiles
    k_fwd_tc<<<grid, TC_THREADS, smem, s>>>(w);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Self-test of the operand layouts, descriptors, the three-part split and the read-back of
// both regions: one CTA multiplies a 128 x 32 A (global, row-major FP32) by the 16 x 32 B
// (row-major FP32) through exactly the split/arrange/issue/commit/drain path of k_fwd_tc.
// The shared allocation is oversized so that no descriptor field, even a misread one, can
// point outside it.
__global__ void __launch_bounds__(TC_THREADS, 1) k_umma_selftest(const float* A, const float* B, float* D, unsigned* err) {
    extern __shared__ unsigned char smem_raw[];
    SmemTC& sm = *reinterpret_cast<SmemTC*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, r = tid & (TM - 1), h = tid >> 7;
    if (tid == 0) {
        mbar_init(&sm.mma_bar[0], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&sm.tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    float x[8];
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        x[q] = A[r * KB + 8 * h + q];
        mx = fmaxf(mx, fabsf(x[q]));
    }
    sm.rowmax[h][r] = mx;
    if (tid < US) {   // species row tid of B on its own grid
        float bm = 0.f;
        for (int c = 0; c < KB; ++c) bm = fmaxf(bm, fabsf(B[tid * KB + c]));
        const Grid g = hi_grid(bm);
        for (int c = 0; c < KB; ++c) {
            float hi, mid, lo;
            split3(B[tid * KB + c], g, hi, mid, lo);
            const int o = (c / 4) * (US * 4) + tid * 4 + (c % 4);
            sm.B[0][o] = hi;
            sm.B[0][US * KB + o] = mid;
            sm.B[0][2 * US * KB + o] = lo;
        }
    }
    __syncthreads();
    const Grid g = hi_grid(fmaxf(fmaxf(sm.rowmax[0][r], sm.rowmax[1][r]), fmaxf(sm.rowmax[2][r], sm.rowmax[3][r])));
    store_split3(sm.A[0][0], x, r, h, g);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sm.tmem_base;
    if (tid == 0) {
        mma_kblock3_species(tbase, tbase + US, sm.A[0][0], sm.B[0]);
        umma_commit(&sm.mma_bar[0]);
    }
    __syncthreads();
    const bool ok = mbar_wait(&sm.mma_bar[0], 0, 2000000000ull);
    tc_fence_after();
    if (ok) {
        if (warp < 8) {
            float acc[8], cmp[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = cmp[q] = 0.f;
            drain_species(tbase, 0, acc, cmp);
            const int row = (warp & 3) * 32 + (tid & 31);
            for (int q = 0; q < 8; ++q) D[row * US + (warp >> 2) * 8 + q] = acc[q] - cmp[q];
        }
    } else if (tid == 0) {
        atomicOr(err, ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, TMEM_COLS);
}

cudaError_t launch_umma_selftest(const float* A, const float* B, float* D, unsigned* err, cudaStream_t s) {
    // oversized: a transposed reading of the descriptor strides stays inside the allocation
    const int smem = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_umma_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_umma_selftest<<<1, TC_THREADS, smem, s>>>(A, B, D, err);
    return cudaGetLastError();
}

}  // namespace bx

namespace bx {

// Waits on an mbarrier that nothing ever arrives on: exercises the bounded-wait path.
__global__ void k_watchdog_selftest(unsigned* err, unsigned long long budget_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (!mbar_wait(&bar, 0, budget_ns) && threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
}

cudaError_t launch_watchdog_selftest(unsigned* err, unsigned long long budget_ns, cudaStream_t s) {
    k_watchdog_selftest<<<1, 32, 0, s>>>(err, budget_ns);
    return cudaGetLastError();
}

}  // namespace bx
