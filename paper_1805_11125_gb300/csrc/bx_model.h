// bx_model.h -- host-side model object shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

// NVTX range around a host-side scope (stage launches, fits): shown by Nsight Systems on the
// host timeline, next to the kernels the scope enqueued
struct BxRange {
    explicit BxRange(const char* name) { nvtxRangePushA(name); }
    ~BxRange() { nvtxRangePop(); }
    BxRange(const BxRange&) = delete;
    BxRange& operator=(const BxRange&) = delete;
};

#include "bx_internal.cuh"

struct FitState;

struct bx_model {
    int n_toys = 0, precision = BX_FP32, cap = 1;
    double band = 8.0;
    unsigned long long watchdog_ns = 2000000000ull;
    cudaStream_t stream = nullptr;
    std::vector<bx::Toy> toys_h;
    std::vector<void*> allocs;   // device allocations owned by the model
    std::vector<void*> pinned;   // pinned host allocations owned by the model
    bx::Work w{};
    int Kmax = 0, Nmax = 0, Mmax = 0, nwmax = 0, nbmax = 0, Lmax = 0, max_tiles = 0, max_cb = 0, P = 0;
    int any_tag = 0, any_cols = 0;   // some toy has a tagged spectrum / an Eq. 4 term
    int is2d = 0;                    // the toys carry 2D histograms (bx_2d.cu path)
    int ncs2d = 0;                   // class-sum rows of the 2D templates (the most over the toys)
    std::vector<int> toy_tmp, toy_cached;
    double* theta_d = nullptr;
    double* nll_d = nullptr;
    double* grad_d = nullptr;
    FitState* fit = nullptr;
    // several energy estimators per dataset (bx_model_create_estimators): toys t E .. t E + E - 1 are
    // the estimators of dataset t; a public item (one dataset at one joint parameter vector of P =
    // Pi + 4 (E - 1) entries) is evaluated as E internal items of Pi = Kmax + 7 parameters each
    int n_est = 1, n_data = 0, Pi = 0;
    double* est_theta = nullptr;        // [cap E][Pi]
    double* est_nll = nullptr;          // [cap E]
    double* est_grad = nullptr;         // [cap E][Pi]
    unsigned char* est_skip = nullptr;  // [cap E]
    // stage timing (bx_model_profile): events recorded between the stage launches
    int prof_on = 0;
    std::vector<cudaEvent_t> prof_ev;   // 6 per recorded evaluation
    size_t prof_used = 0;
};

enum { BX_STAGES = 5 };   // prep, forward, assembly, adjoint, gather

int bx_set_error(int code, const char* fmt, ...);
int bx_set_items(bx_model* m, int n, const int* toy_idx);
int bx_enqueue_eval(bx_model* m, int n, const double* theta_dev, int tstride, int want_grad, int want_mu,
                    double* nll_dev, double* grad_dev);
int bx_take_device_error(bx_model* m);
// parameters of public item rows of dataset t (K_t + 7 + 4 (E - 1))
int bx_public_P(const bx_model* m, int t);
// forward tile shapes the model can run (the FP32 forward: 128- or 64-row CTAs), and the choice
int bx_fwd_tile_variants(const bx_model* m);
void bx_set_fwd_tile(bx_model* m, int variant);
void bx_fit_free(bx_model* m);
