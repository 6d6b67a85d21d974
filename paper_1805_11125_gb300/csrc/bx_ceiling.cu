// bx_ceiling.cu -- input-free microkernels that measure the ceilings the roofline of the
// likelihood kernels is taken against (the paper has no counterpart; these are measurement
// tools of the build).
//
//   CEIL_RESP       the FP32 bin-mass routine of the forward (resp_shape32, the series branch
//                   the forward takes for in-band entries) over a band of synthetic columns:
//                   the most in-band response entries per second this GPU can generate;
//   CEIL_RESP_ACC   the same routine plus the forward's per-entry accumulation (two
//                   Kahan-compensated row sums, one column-sum FMA): the per-entry work of
//                   the rate-first forward with nothing else (no staging, masks or stores);
//   CEIL_FMA64      FP64 FMA throughput (8 independent chains per thread);
//   CEIL_FMA32      FP32 FMA throughput (8 independent chains per thread).
//
// Every kernel runs a grid of whole waves (SMs x resident blocks per SM), reads nothing,
// and writes one value per thread so that no work can be dropped.  The column parameters of
// CEIL_RESP are those of a Gaussian of sigma 20..35 npe on 1-npe bins, its band +-8.7 sigma
// (512 rows), so every entry takes the same branch as an in-band entry of the forward.
#include <cuda_runtime.h>

#include <math.h>

#include "bx_internal.cuh"
#include "bx_model.h"
#include "bx_resp.cuh"

namespace bx {

constexpr int CEIL_THREADS = 256;
constexpr int CEIL_ROWS = 512;   // rows of one synthetic column's band
constexpr int CEIL_CHAINS = 8;

__device__ __forceinline__ void ceil_kahan(float& acc, float& cmp, float a, float b) {
    const float y = fmaf(a, b, -cmp);
    const float t = __fadd_rn(acc, y);
    cmp = __fsub_rn(__fsub_rn(t, acc), y);
    acc = t;
}

template <bool ACC>
__global__ void __launch_bounds__(CEIL_THREADS) k_ceiling_resp(int reps, float* sink) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    // one synthetic column per thread: sigma in npe, mean mu/w, its FP32 generator constants
    const float sig = 20.0f + (float)(gid & 15);
    const float hs = 0.84932180028801904f / sig;              // (w / sigma) S_EX2, w = 1
    const float muw = 1000.25f + 0.37f * (float)(gid & 63);
    const float fl = floorf(muw);
    const float4 cf = make_float4(fl, (0.5f - (muw - fl)) * hs, hs, 0.0f);
    const float kk = 0.38729833462f * hs;                      // sqrt(3/5) / 2 hs
    ColG cg;
    cg.kap = 1.38629436112f * kk;                              // 2 ln2 kk
    cg.Ck2 = 2.0f * exp2f(-kk * kk);
    cg.c_lo = 0.0f;
    cg.A = 1.0f;
    const float S1 = 0.75f, S2 = 0.25f, G = 0.5f;
    float acc = 0.f, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, col = 0.f;
    const float row0 = fl - (float)(CEIL_ROWS / 2);
    for (int rep = 0; rep < reps; ++rep) {
        const float base = row0 + (float)(rep % 3);            // the band moves by a row or two per pass
#pragma unroll 4
        for (int r = 0; r < CEIL_ROWS; ++r) {
            const float R = resp_shape32<true>(base + (float)r, cf, cg);
            if (ACC) {
                ceil_kahan(s1, c1, R, S1);
                ceil_kahan(s2, c2, R, S2);
                col = fmaf(R, G, col);
            } else {
                acc += R;
            }
        }
    }
    sink[gid] = ACC ? (s1 + c1) + (s2 + c2) + col : acc;
}

__global__ void __launch_bounds__(CEIL_THREADS) k_ceiling_fma64(int reps, float* sink) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    double x[CEIL_CHAINS];
#pragma unroll
    for (int c = 0; c < CEIL_CHAINS; ++c) x[c] = 1.0 + 1e-3 * (gid + c);
    const double a = 0.999999, b = 1e-7;
    for (int rep = 0; rep < reps; ++rep)
#pragma unroll 16
        for (int j = 0; j < 64; ++j)
#pragma unroll
            for (int c = 0; c < CEIL_CHAINS; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CEIL_CHAINS; ++c) s += x[c];
    sink[gid] = (float)s;
}

__global__ void __launch_bounds__(CEIL_THREADS) k_ceiling_fma32(int reps, float* sink) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    float x[CEIL_CHAINS];
#pragma unroll
    for (int c = 0; c < CEIL_CHAINS; ++c) x[c] = 1.0f + 1e-3f * (float)(gid + c);
    const float a = 0.999999f, b = 1e-7f;
    for (int rep = 0; rep < reps; ++rep)
#pragma unroll 16
        for (int j = 0; j < 64; ++j)
#pragma unroll
            for (int c = 0; c < CEIL_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CEIL_CHAINS; ++c) s += x[c];
    sink[gid] = s;
}

}  // namespace bx

using namespace bx;

template <typename K>
static int ceiling_run(K kern, int reps, cudaStream_t s, double units_per_thread_rep, double* ms, double* units) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CEIL_THREADS, 0);
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "bx_ceiling: %s", cudaGetErrorString(e));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    float* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&sink, sizeof(float) * (size_t)blocks * CEIL_THREADS);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float t = 0.f;
    if (e == cudaSuccess) {
        kern<<<blocks, CEIL_THREADS, 0, s>>>(reps > 4 ? reps / 4 : 1, sink);   // warm-up (clocks, caches)
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) {
        kern<<<blocks, CEIL_THREADS, 0, s>>>(reps, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "bx_ceiling: %s", cudaGetErrorString(e));
    *ms = t;
    *units = units_per_thread_rep * (double)reps * (double)blocks * CEIL_THREADS;
    return BX_OK;
}

extern "C" int bx_ceiling(int which, int reps, void* cuda_stream, double* ms, double* units) {
    if (!ms || !units) return bx_set_error(BX_EINVAL, "bx_ceiling: NULL output");
    if (reps < 1 || reps > 1 << 20) return bx_set_error(BX_EINVAL, "bx_ceiling: reps %d out of [1, 2^20]", reps);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    switch (which) {
        case BX_CEIL_RESP: return ceiling_run(k_ceiling_resp<false>, reps, s, CEIL_ROWS, ms, units);
        case BX_CEIL_RESP_ACC: return ceiling_run(k_ceiling_resp<true>, reps, s, CEIL_ROWS, ms, units);
        case BX_CEIL_FMA64: return ceiling_run(k_ceiling_fma64, reps, s, 2.0 * 64 * CEIL_CHAINS, ms, units);
        case BX_CEIL_FMA32: return ceiling_run(k_ceiling_fma32, reps, s, 2.0 * 64 * CEIL_CHAINS, ms, units);
        default: return bx_set_error(BX_EINVAL, "bx_ceiling: unknown ceiling %d", which);
    }
}
