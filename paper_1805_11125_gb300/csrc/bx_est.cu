// bx_est.cu -- several energy estimators of one dataset, fitted jointly.
//
// The paper's Sec. 3 names three energy estimators of the same events -- the charge, the
// number of detected photons and the number of fired channels -- each an observable N_x with
// its own response R_x of Eq. 1.  Reading: the estimators share the deposited-energy spectra
// and what acts on them before the detector response (the rates, the Birks constant kB, the
// pile-up probability eps, the radial scale s_r); each has its own response parameters (LY, a,
// b, c), binning, window, random-trigger spectrum and data, and the joint -lnL is the sum of
// the estimators' -lnL.  The joint parameter vector of a dataset with K species is
//   [r_0 .. r_{K-1}, LY_0, a_0, b_0, c_0, kB, eps, s_r, LY_1, a_1, b_1, c_1, ..., c_{E-1}]
// (P = K + 7 + 4 (E - 1); E = 1 is the single model).  One public evaluation item becomes E
// internal items, evaluated by the regular kernels in the same batch (estimator e of item j is
// internal item j E + e, at [r, LY_e, a_e, b_e, c_e, kB, eps, s_r]); k_est_join sums their -lnL
// and maps their gradients back onto the joint vector.
#include <cuda_runtime.h>

#include "bx_internal.cuh"

namespace bx {

// Internal parameter rows (and skip flags) of the n E internal items.
__global__ void k_est_split(const double* theta, int tstride, int n, int E, const Toy* toys, const int* toy_of,
                            const unsigned char* skip, double* th_int, int Pi, unsigned char* skip_int) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;   // internal item
    if (j >= n * E) return;
    const int pub = j / E, e = j % E;
    const int K = toys[toy_of[j]].K;
    const double* src = theta + (size_t)pub * tstride;
    double* dst = th_int + (size_t)j * Pi;
    const int so = e == 0 ? K : K + 7 + 4 * (e - 1);   // LY_e, a_e, b_e, c_e in the joint row
    for (int q = 0; q < Pi; ++q) {
        double v = 0.0;
        if (q < K) v = src[q];                      // rates
        else if (q < K + 4) v = src[so + q - K];    // the estimator's response parameters
        else if (q < K + 7) v = src[q];             // kB, eps, s_r
        dst[q] = v;
    }
    if (skip_int) skip_int[j] = skip ? skip[pub] : 0;
}

// Joint -lnL (the sum over the estimators) and gradient of every public item.
__global__ void k_est_join(const double* nll_int, const double* grad_int, int Pi, int n, int E, const Toy* toys,
                           const int* toy_of, double* nll, double* grad, int P, int want_grad) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;   // public item
    if (j >= n) return;
    const int K = toys[toy_of[(size_t)j * E]].K;
    double f = 0.0;
    for (int e = 0; e < E; ++e) f += nll_int[(size_t)j * E + e];
    nll[j] = f;
    if (!want_grad) return;
    double* g = grad + (size_t)j * P;
    for (int q = 0; q < P; ++q) g[q] = 0.0;
    for (int e = 0; e < E; ++e) {
        const double* ge = grad_int + ((size_t)j * E + e) * Pi;
        const int so = e == 0 ? K : K + 7 + 4 * (e - 1);
        for (int k = 0; k < K; ++k) g[k] += ge[k];
        for (int q = 0; q < 4; ++q) g[so + q] += ge[K + q];
        for (int q = 4; q < 7; ++q) g[K + q] += ge[K + q];
    }
}

cudaError_t launch_est_split(const double* theta, int tstride, int n, int E, const Toy* toys, const int* toy_of,
                             const unsigned char* skip, double* th_int, int Pi, unsigned char* skip_int, cudaStream_t s) {
    const int ni = n * E;
    k_est_split<<<(ni + 127) / 128, 128, 0, s>>>(theta, tstride, n, E, toys, toy_of, skip, th_int, Pi, skip_int);
    return cudaGetLastError();
}

cudaError_t launch_est_join(const double* nll_int, const double* grad_int, int Pi, int n, int E, const Toy* toys,
                            const int* toy_of, double* nll, double* grad, int P, int want_grad, cudaStream_t s) {
    k_est_join<<<(n + 127) / 128, 128, 0, s>>>(nll_int, grad_int, Pi, n, E, toys, toy_of, nll, grad, P, want_grad);
    return cudaGetLastError();
}

}  // namespace bx
