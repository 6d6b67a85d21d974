// bx_fwd_tc.cu -- Eq. 1 forward on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Unit = (row tile of TM = 128 output bins, item); one CTA of 128 threads, thread = bin.
// For every k-block of KB = 32 true-energy columns of the tile's band:
//   * one thread starts a TMA bulk copy of the k-block's species tile (TF32 hi | lo of
//     s_k[i], pre-arranged in the UMMA K-major layout at model creation);
//   * all threads generate the 128 x 32 response tile in FP32 -- the bin mass of the
//     Gaussian by 3-point Gauss-Legendre quadrature of its density (no difference of
//     CDFs, hence no cancellation) times the FP64-derived column normalisation -- split it
//     into TF32 hi and lo and store both in shared memory in the UMMA K-major layout;
//   * one thread issues D += A_hi B_hi + A_hi B_lo + A_lo B_hi (M = 128, N = 16, K = 8
//     per instruction) into one of NACC rotating FP32 accumulators in tensor memory and
//     commits to the stage's mbarrier.
// Two stages alternate, so the generation of k-block j overlaps the MMAs of j - 1.  The
// epilogue sums the accumulators in FP64 and stores v[m][k] as FP32.
// Every wait is bounded by the watchdog budget; on expiry the CTA records ERR_TIMEOUT,
// waits (bounded, at least 2 s) for its own bulk copies and MMAs, frees its tensor memory
// and returns.
#include <math.h>

#include "bx_internal.cuh"

namespace bx {

constexpr int R_FLOATS = TM * KB;          // one response tile (hi or lo)
constexpr int S_FLOATS = 2 * US * KB;      // species tile hi | lo
constexpr uint32_t S_BYTES = S_FLOATS * 4;
constexpr uint32_t TMEM_COLS = NACC * US;  // 64

struct __align__(128) SmemTC {
    float Rhi[2][R_FLOATS];
    float Rlo[2][R_FLOATS];
    float S[2][S_FLOATS];
    float4 colp[2][KB];
    float colA[2][KB];
    uint64_t mma_bar[2];
    uint64_t s_bar[2];
    uint32_t tmem_base;
    int abort;
};

// Response entry of output bin `mf` (row index as float) and one column, FP32, with the
// hardware ex2 approximation (the tensor-core variant; see bx_resp.cuh for the exact form).
__device__ __forceinline__ float resp_f32(float mf, float4 cp, float A) {
    const float t0 = fmaf(mf - cp.x, cp.z, cp.y);
    const float tm = fmaf(-GL_NODE_HALF, cp.z, t0);
    const float tp = fmaf(GL_NODE_HALF, cp.z, t0);
    const float p0 = ex2_approx(-(t0 * t0));
    const float pm = ex2_approx(-(tm * tm));
    const float pp = ex2_approx(-(tp * tp));
    return A * fmaf(GL_W_OUT, pm + pp, GL_W_MID * p0);
}

// Generate this thread's row of a response tile (KB columns) into the hi/lo tiles.
// Layout: element (row r, col c) at float (c/4)*TM*4 + r*4 + c%4.
__device__ __forceinline__ void gen_row(float* Rhi, float* Rlo, const float4* colp, const float* colA, int r,
                                        float mf) {
#pragma unroll
    for (int c4 = 0; c4 < KB / 4; ++c4) {
        float4 hi, lo;
        float x;
        x = resp_f32(mf, colp[c4 * 4 + 0], colA[c4 * 4 + 0]); hi.x = tf32_rna(x); lo.x = tf32_rna(x - hi.x);
        x = resp_f32(mf, colp[c4 * 4 + 1], colA[c4 * 4 + 1]); hi.y = tf32_rna(x); lo.y = tf32_rna(x - hi.y);
        x = resp_f32(mf, colp[c4 * 4 + 2], colA[c4 * 4 + 2]); hi.z = tf32_rna(x); lo.z = tf32_rna(x - hi.z);
        x = resp_f32(mf, colp[c4 * 4 + 3], colA[c4 * 4 + 3]); hi.w = tf32_rna(x); lo.w = tf32_rna(x - hi.w);
        reinterpret_cast<float4*>(Rhi)[c4 * TM + r] = hi;
        reinterpret_cast<float4*>(Rlo)[c4 * TM + r] = lo;
    }
}

// Issue the split-precision MMAs of one k-block into accumulator `dslot`.
__device__ __forceinline__ void issue_kblock(uint32_t dslot, const float* Rhi, const float* Rlo, const float* S,
                                             bool accumulate) {
    constexpr uint32_t idesc = umma_idesc_tf32(TM, US);
    const uint32_t a_hi = smem_u32(Rhi), a_lo = smem_u32(Rlo);
    const uint32_t b_hi = smem_u32(S), b_lo = b_hi + US * KB * 4;
#pragma unroll
    for (int q = 0; q < KB / 8; ++q) {
        // one K = 8 step spans two core-matrix columns
        const uint64_t ahi = umma_desc(a_hi + q * 2 * (TM * 16), TM * 16, 128);
        const uint64_t alo = umma_desc(a_lo + q * 2 * (TM * 16), TM * 16, 128);
        const uint64_t bhi = umma_desc(b_hi + q * 2 * (US * 16), US * 16, 128);
        const uint64_t blo = umma_desc(b_lo + q * 2 * (US * 16), US * 16, 128);
        umma_tf32(dslot, ahi, bhi, idesc, (accumulate || q > 0) ? 1u : 0u);
        umma_tf32(dslot, ahi, blo, idesc, 1u);
        umma_tf32(dslot, alo, bhi, idesc, 1u);
    }
}

__global__ void __launch_bounds__(TM, 3) k_fwd_tc(Work w) {
    extern __shared__ unsigned char smem_raw[];
    SmemTC& sm = *reinterpret_cast<SmemTC*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    // 1D item-major grid (a y dimension would cap the batch at 65535 items)
    const int tile = blockIdx.x % w.max_tiles, item = blockIdx.x / w.max_tiles, tid = threadIdx.x, warp = tid >> 5;
    const Toy& T = w.toys[w.toy_of[item]];
    if (tile >= T.n_tiles || w.status[item]) return;
    const int m0 = tile * TM, M = T.M;
    const int2 cr = w.tile_cols[(size_t)item * MAX_TILES + tile];
    float* vrow = static_cast<float*>(w.v) + ((size_t)item * w.Mpad + m0 + tid) * US;
    const bool row_ok = m0 + tid < M;
    const int kb0 = cr.x < cr.y ? cr.x / KB : 0;
    const int nblk = cr.x < cr.y ? (cr.y - 1) / KB + 1 - kb0 : 0;
    if (nblk <= 0) {
        if (row_ok) {
#pragma unroll
            for (int k = 0; k < US; k += 4) *reinterpret_cast<float4*>(vrow + k) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    const float4* colf = w.colf + (size_t)item * w.Npad + (size_t)kb0 * KB;
    const ColG* colg = w.colg + (size_t)item * w.Npad + (size_t)kb0 * KB;
    const float* Sg = T.S_tiles + (size_t)kb0 * S_FLOATS;

    if (tid == 0) {
        mbar_init(&sm.mma_bar[0], 1);
        mbar_init(&sm.mma_bar[1], 1);
        mbar_init(&sm.s_bar[0], 1);
        mbar_init(&sm.s_bar[1], 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&sm.tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
    float preA = 0.f;
    if (tid < KB) {
        sm.colp[0][tid] = colf[tid];
        sm.colA[0][tid] = colg[tid].A;
        if (nblk > 1) {
            pre = colf[KB + tid];
            preA = colg[KB + tid].A;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sm.tmem_base;
    if (tid == 0) {
        mbar_arrive_expect_tx(&sm.s_bar[0], S_BYTES);
        bulk_g2s(sm.S[0], Sg, S_BYTES, &sm.s_bar[0]);
    }
    const float mf = (float)(m0 + tid);
    // thread 0 bookkeeping: bulk copies issued / waited for, k-blocks committed
    int s_issued = 1, s_waited = 0, committed = 0;

    for (int it = 0; it < nblk; ++it) {
        const int s = it & 1;
        if (it >= 2 && !mbar_wait(&sm.mma_bar[s], ((it - 2) >> 1) & 1, w.watchdog_ns)) atomicOr(&sm.abort, 1);
        __syncthreads();
        if (sm.abort) break;
        if (tid == 0 && it >= 1) {
            mbar_arrive_expect_tx(&sm.s_bar[s], S_BYTES);
            bulk_g2s(sm.S[s], Sg + (size_t)it * S_FLOATS, S_BYTES, &sm.s_bar[s]);
            ++s_issued;
        }
        gen_row(sm.Rhi[s], sm.Rlo[s], sm.colp[s], sm.colA[s], tid, mf);
        if (tid < KB && it + 1 < nblk) {
            sm.colp[s ^ 1][tid] = pre;
            sm.colA[s ^ 1][tid] = preA;
            if (it + 2 < nblk) {
                pre = colf[(size_t)(it + 2) * KB + tid];
                preA = colg[(size_t)(it + 2) * KB + tid].A;
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            if (!mbar_wait(&sm.s_bar[s], (it >> 1) & 1, w.watchdog_ns)) {
                atomicOr(&sm.abort, 1);
            } else {
                ++s_waited;
                issue_kblock(tbase + (uint32_t)((it % NACC) * US), sm.Rhi[s], sm.Rlo[s], sm.S[s], it >= NACC);
                umma_commit(&sm.mma_bar[s]);
                ++committed;
            }
        }
    }
    // Drain: every bulk copy and MMA of this CTA must have landed before the CTA frees its
    // tensor memory or exits.  Thread 0 waits for its outstanding copies; the last commit
    // completes after every earlier MMA of the issuing thread.  Bounded by CLEANUP_NS.
    constexpr unsigned long long CLEANUP_NS = 2000000000ull;
    if (tid == 0) {
        bool drained = true;
        for (int j = s_waited; j < s_issued; ++j)
            drained &= mbar_wait(&sm.s_bar[j & 1], (j >> 1) & 1, CLEANUP_NS);
        if (!drained) atomicOr(&sm.abort, 1);
        sm.tmem_base = tbase;
        // publish the number of committed k-blocks for the other threads
        sm.abort |= committed << 8;
    }
    __syncthreads();
    const int ncommit = sm.abort >> 8;
    const bool aborted = (sm.abort & 0xff) != 0;
    bool done = true;
    if (ncommit > 0) {
        const int last = ncommit - 1;
        done = mbar_wait(&sm.mma_bar[last & 1], (last >> 1) & 1,
                        w.watchdog_ns > CLEANUP_NS ? w.watchdog_ns : CLEANUP_NS);
    }
    tc_fence_after();
    if (aborted || !done || ncommit != nblk) {
        if (tid == 0) atomicOr(w.err, ERR_TIMEOUT);
    } else {
        double acc[US];
#pragma unroll
        for (int k = 0; k < US; ++k) acc[k] = 0.0;
        const int nslot = nblk < NACC ? nblk : NACC;
        for (int sl = 0; sl < nslot; ++sl) {
            float r[US];
            tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sl * US), r);
#pragma unroll
            for (int k = 0; k < US; ++k) acc[k] += (double)r[k];
        }
        if (row_ok) {
#pragma unroll
            for (int k = 0; k < US; k += 4)
                *reinterpret_cast<float4*>(vrow + k) =
                    make_float4((float)acc[k], (float)acc[k + 1], (float)acc[k + 2], (float)acc[k + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, TMEM_COLS);
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
    k_fwd_tc<<<grid, TM, smem, s>>>(w);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Self-test of the operand layouts, descriptors and accumulator read-back: one CTA
// multiplies a 128 x 32 A (global, row-major FP32) by the 16 x 32 B (row-major FP32)
// through exactly the split/arrange/issue/commit/read path of k_fwd_tc.  The shared
// allocation is oversized so that no descriptor field, even a misread one, can point
// outside it.
__global__ void __launch_bounds__(TM, 1) k_umma_selftest(const float* A, const float* B, float* D, unsigned* err) {
    extern __shared__ unsigned char smem_raw[];
    SmemTC& sm = *reinterpret_cast<SmemTC*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&sm.mma_bar[0], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&sm.tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    // A row tid -> hi/lo tiles
    for (int c4 = 0; c4 < KB / 4; ++c4) {
        float4 hi, lo;
        const float* a = A + tid * KB + c4 * 4;
        hi.x = tf32_rna(a[0]); lo.x = tf32_rna(a[0] - hi.x);
        hi.y = tf32_rna(a[1]); lo.y = tf32_rna(a[1] - hi.y);
        hi.z = tf32_rna(a[2]); lo.z = tf32_rna(a[2] - hi.z);
        hi.w = tf32_rna(a[3]); lo.w = tf32_rna(a[3] - hi.w);
        reinterpret_cast<float4*>(sm.Rhi[0])[c4 * TM + tid] = hi;
        reinterpret_cast<float4*>(sm.Rlo[0])[c4 * TM + tid] = lo;
    }
    for (int j = tid; j < US * KB; j += TM) {
        const int n = j / KB, c = j % KB;
        const float b = B[j], hi = tf32_rna(b);
        sm.S[0][(c / 4) * (US * 4) + n * 4 + (c % 4)] = hi;
        sm.S[0][US * KB + (c / 4) * (US * 4) + n * 4 + (c % 4)] = tf32_rna(b - hi);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sm.tmem_base;
    if (tid == 0) {
        issue_kblock(tbase, sm.Rhi[0], sm.Rlo[0], sm.S[0], false);
        umma_commit(&sm.mma_bar[0]);
    }
    __syncthreads();
    const bool ok = mbar_wait(&sm.mma_bar[0], 0, 2000000000ull);
    tc_fence_after();
    if (ok) {
        float r[US];
        tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16), r);
        for (int k = 0; k < US; ++k) D[tid * US + k] = r[k];
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
    k_umma_selftest<<<1, TM, smem, s>>>(A, B, D, err);
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
