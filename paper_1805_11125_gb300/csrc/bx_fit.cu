// bx_fit.cu -- batched fits driven by the adjoint gradient (the minimisation of Sec. 4,
// done there by TMinuit with numerical derivatives of -lnL).
//
// Every fit owns a block of S = NLS + 2P evaluation slots in the batch and a state on the
// device.  One iteration = one batched -lnL + gradient evaluation of every slot in use
// (the regular evaluation kernels; unused slots are skipped) followed by k_fit, one thread
// per fit, which advances a damped Newton state machine:
//   START  slot 0 holds the starting point: accept it, go to HESS;
//   HESS   slots NLS + 2a, NLS + 2a + 1 hold theta +- h e_j for the a-th free parameter j:
//          the Hessian columns come from central differences of the exact gradient, all
//          in one launch; it is inverted on the free set as the Cholesky factor of the
//          diagonally scaled matrix D H D + mu I with the smallest Levenberg damping mu that
//          makes it positive definite; EDM = g^T V g / 2 of the fresh, least-damped matrix
//          decides convergence; otherwise go to LS;
//   LS     slots 0..NLS-1 hold theta + 2^-k d (projected on the bounds), all evaluated in one
//          launch; the largest step satisfying the Armijo condition is accepted (below the
//          FP32 noise floor of -lnL an undamped full step is accepted as is) and HESS
//          follows; if none qualifies the damping is raised and LS repeats;
//   DONE   converged (OK), evaluation budget exhausted or damping runaway (ENOTCONV),
//          -lnL = +inf at the start (EDOMAIN).
// The likelihood is non-convex away from its optimum and ill-conditioned near it (light
// yield, Birks and resolution parameters are nearly degenerate), so the curvature is
// re-measured at every iterate instead of being accumulated by rank-two updates; the slot
// blocks make that a single launch, and a whole Newton iteration costs two.  Box bounds
// are handled by projection; parameters pinned at a bound with the gradient pointing out
// are excluded from the step.  The iterations are captured once into a CUDA graph
// (iters_per_launch iterations per replay); the host replays it until no fit is active,
// reading one counter per replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "bx_internal.cuh"
#include "bx_model.h"

using namespace bx;

namespace {

constexpr int NLS = 8;   // line-search trial steps per iteration: 1, 1/2, ..., 1/128
// parameters of a fit: K + 7, plus 4 per further energy estimator
constexpr int PFMAX = KMAX + 7 + 4 * (MAX_EST - 1);

enum { PH_START = 0, PH_HESS = 1, PH_LS = 2, PH_DONE = 3 };

// Predicted decrease below which FP32 evaluations cannot confirm a decrease of -lnL (their
// -lnL carries ~5e-5 of rounding noise): an undamped full Newton step is then accepted
// without the sufficient-decrease test, provided -lnL does not rise by more than the noise.
constexpr double EDM_NOISE = 5e-5;
// Largest damping (scaled units) with which a fresh Hessian may declare convergence
// (FitCtl::mu_conv): a damping mu lowers the EDM along a direction of curvature lambda < mu
// by lambda / mu.  With FP64 evaluations mu <= 1e-2 keeps the distance missed that way below
// ~0.01 sigma for the weakest curvature of these models (~6e-6 scaled) at tol_edm = 1e-8.
// FP32 gradients make the finite-difference Hessian noisy in that direction and need up to
// 1e-1; their -lnL noise (~5e-5) limits the optimum to ~0.01 sigma in any case, and an FP64
// fit started from the FP32 optimum polishes it in a few iterations.
constexpr double MU_CONV_FP64 = 1e-2, MU_CONV_FP32 = 1e-1;
// EDM floor of FP32 evaluations: their gradient noise (~1e-5 in scaled units) projected on
// the weakest direction (scaled curvature ~3e-5) gives EDM ~ 1e-6 .. 1e-5 at the optimum,
// i.e. a distance below ~0.005 sigma; FP32 fits use max(tol_edm, EDM_FLOOR_FP32).
constexpr double EDM_FLOOR_FP32 = 1e-5;

// Finite-difference steps of the Hessian.  FP64 fits step hrel |theta_j|.  FP32 fits step
// HSIG_FP32 conditional standard deviations 1 / sqrt(H_jj) of the last Hessian once one exists.
// Relative steps span ~1e-3 to ~10 sigma across these parameters, and where the step was a
// small fraction of sigma the FP32 gradient noise, divided by the step, swamped the weakest
// directions.  Measured over 11 FP32 fits from 10% starts, 10 converge with 1 sigma, 9 with
// 0.3 sigma and 8 with relative steps.  Steps stay below half the parameter's magnitude (a
// rate stepped to zero could empty a bin).
constexpr double HSIG_FP32 = 1.0;

// Trust region of the response, pile-up and radial parameters.  Far from the optimum the Newton
// step of these nearly degenerate parameters can be many times their value (the light yield,
// the resolution terms and kB trade off against each other), and a line search along it may
// accept a point from which the fit runs onto the bounds: a 5%-off start of the small joint
// model walked the resolution term b to 25 times its value with four parameters held at bounds.
// Near the optimum every step is well inside the region (a few standard deviations at most).
constexpr double TR_REL = 0.5, TR_SIG = 2.0;

struct FitCtl {
    int phase, iters, evals, status, max_evals, fails, n_bound;
    double edm, edm0, tol, mu_min, mu_used, hrel, mu_conv, hsig, mu_fresh;
};

struct FitDev {
    int n, P, S;
    const int* Pf;          // per fit: parameters of its dataset's row (K_t + 7 + 4 (E - 1))
    const int* Kf;          // per fit: rates (K_t), the parameters before the trust-region ones
    double *theta, *g, *f;  // accepted state per fit
    double *H, *V, *d;      // per fit
    double *lo, *hi;        // per fit
    unsigned char* fr;      // per fit
    double *tt, *ft, *gt;   // per slot: evaluation input and outputs
    unsigned char* skip;    // per slot
    FitCtl* ctl;
    int* active;
};

#define IDX(i, j) ((i) * P + (j))

// V <- (H + damping)^-1 on the active set of the first n parameters (row stride P):
// Cholesky of C = D H D + mu I (D = |diag H|^-1/2) for the smallest mu in
// {mu_min, 10 mu_min, ...} (mu_min = 0 tries the undamped matrix first, then 1e-6).
// Returns the mu used, or -1 when even mu = 1e8 fails.
__device__ double damped_inverse(const double* H, const unsigned char* act, int n, int P, double mu_min, double* V,
                                 double* L) {
    int idx[PFMAX], nf = 0;
    double D[PFMAX];
    for (int i = 0; i < n; ++i)
        if (act[i]) {
            const double h = fabs(H[IDX(i, i)]);
            D[nf] = (h > 0.0 && isfinite(h)) ? 1.0 / sqrt(h) : 1.0;
            idx[nf++] = i;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[IDX(i, j)] = 0.0;
    double mu = mu_min;
    for (int attempt = 0; attempt < 40; ++attempt, mu = (mu == 0.0 ? 1e-6 : mu * 10.0)) {
        if (mu > 1e8) return -1.0;
        bool ok = true;
        for (int a = 0; a < nf && ok; ++a)
            for (int b = 0; b <= a; ++b) {
                const int ia = idx[a], ib = idx[b];
                double c = 0.5 * (H[IDX(ia, ib)] + H[IDX(ib, ia)]) * D[a] * D[b] + (a == b ? mu : 0.0);
                for (int k = 0; k < b; ++k) c -= L[a * nf + k] * L[b * nf + k];
                if (a == b) {
                    if (!(c > 0.0) || !isfinite(c)) { ok = false; break; }
                    L[a * nf + a] = sqrt(c);
                } else {
                    L[a * nf + b] = c / L[b * nf + b];
                }
            }
        if (!ok) continue;
        double col[PFMAX];
        for (int c = 0; c < nf; ++c) {
            for (int i = 0; i < nf; ++i) {
                double t = (i == c) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) t -= L[i * nf + k] * col[k];
                col[i] = t / L[i * nf + i];
            }
            for (int i = nf - 1; i >= 0; --i) {
                double t = col[i];
                for (int k = i + 1; k < nf; ++k) t -= L[k * nf + i] * col[k];
                col[i] = t / L[i * nf + i];
            }
            for (int i = 0; i < nf; ++i) V[IDX(idx[i], idx[c])] = D[i] * col[i] * D[c];
        }
        return mu;
    }
    return -1.0;
}

__global__ void k_fit(FitDev F) {
    const int jf = blockIdx.x * blockDim.x + threadIdx.x;
    if (jf >= F.n) return;
    const int P = F.P, S = F.S;
    FitCtl c = F.ctl[jf];
    if (c.phase == PH_DONE) return;
    const size_t s0 = (size_t)jf * S;   // first slot of this fit
    const int Pt = F.Pf[jf], Kt = F.Kf[jf];
    double* th = F.theta + (size_t)jf * P;
    double* g = F.g + (size_t)jf * P;
    double* V = F.V + (size_t)jf * P * P;
    double* H = F.H + (size_t)jf * P * P;
    double* d = F.d + (size_t)jf * P;
    const double* lo = F.lo + (size_t)jf * P;
    const double* hi = F.hi + (size_t)jf * P;
    const unsigned char* fr = F.fr + (size_t)jf * P;
    auto slot_t = [&](int k) { return F.tt + (s0 + k) * P; };
    auto slot_g = [&](int k) { return F.gt + (s0 + k) * P; };
    bool to_hess = false, newdir = false, fresh = false;

    if (c.phase == PH_START) {
        const double f0 = F.ft[s0];
        for (int i = 0; i < Pt; ++i) { th[i] = slot_t(0)[i]; g[i] = slot_g(0)[i]; }
        F.f[jf] = f0;
        if (!isfinite(f0)) { c.phase = PH_DONE; c.status = BX_EDOMAIN; }
        else to_hess = true;
    } else if (c.phase == PH_HESS) {
        int a = 0;
        for (int j = 0; j < Pt; ++j) {
            if (!fr[j]) continue;
            const double* gp = slot_g(NLS + 2 * a);
            const double* gm = slot_g(NLS + 2 * a + 1);
            const double up = slot_t(NLS + 2 * a)[j], dn = slot_t(NLS + 2 * a + 1)[j];
            for (int i = 0; i < Pt; ++i) H[IDX(i, j)] = fr[i] ? (gp[i] - gm[i]) / (up - dn) : 0.0;
            ++a;
        }
        newdir = fresh = true;
    } else if (c.phase == PH_LS) {
        int acc = -1;
        for (int k = 0; k < NLS && acc < 0; ++k) {
            const double fk = F.ft[s0 + k];
            if (!isfinite(fk)) continue;
            double gs = 0.0;
            const double* tk = slot_t(k);
            for (int i = 0; i < Pt; ++i) gs += g[i] * (tk[i] - th[i]);
            const bool noise_floor = k == 0 && c.mu_used <= c.mu_conv && c.edm0 < EDM_NOISE &&
                                     fk <= F.f[jf] + 2.0 * EDM_NOISE;
            if (fk <= F.f[jf] + 1e-4 * gs || noise_floor) acc = k;
        }
        if (acc >= 0) {
            for (int i = 0; i < Pt; ++i) { th[i] = slot_t(acc)[i]; g[i] = slot_g(acc)[i]; }
            F.f[jf] = F.ft[s0 + acc];
            c.iters++;
            c.mu_min = 0.0;
            to_hess = true;
        } else {
            c.fails++;
            c.mu_min = c.mu_used > 0.0 ? c.mu_used * 1e3 : 1e-3;
            newdir = true;
        }
    }
    if (newdir) {
        unsigned char act[PFMAX];
        for (int i = 0; i < Pt; ++i)
            act[i] = fr[i] && !((th[i] <= lo[i] && g[i] > 0.0) || (th[i] >= hi[i] && g[i] < 0.0));
        double L[PFMAX * PFMAX];
        const double mu = damped_inverse(H, act, Pt, P, fresh ? 0.0 : c.mu_min, V, L);
        double gd = 0.0;
        if (mu >= 0.0) {
            for (int i = 0; i < Pt; ++i) {
                double t = 0.0;
                if (act[i])
                    for (int k = 0; k < Pt; ++k) t -= V[IDX(i, k)] * g[k];
                d[i] = t;
                gd += g[i] * t;
            }
        }
        if (mu < 0.0) {
            c.phase = PH_DONE;
            c.status = BX_ENOTCONV;
        } else {
            c.mu_used = mu;
            c.edm = -0.5 * gd;
            if (fresh) {
                c.edm0 = c.edm;
                c.mu_fresh = mu;
                int nb = 0;
                for (int i = 0; i < Pt; ++i) nb += (fr[i] && !act[i]) ? 1 : 0;
                c.n_bound = nb;
            }
            if (fresh && c.edm < c.tol && mu <= c.mu_conv) {
                c.phase = PH_DONE;
                c.status = BX_OK;
            } else {
                c.phase = PH_LS;
                // trust region of the response, pile-up and radial parameters (everything after the
                // rates): a trial step moves none of them by more than TR_REL of its magnitude or
                // TR_SIG of its standard deviation under the current Hessian, whichever is larger
                double amax = 1.0;
                for (int i = Kt; i < Pt; ++i)
                    if (act[i] && d[i] != 0.0) {
                        const double v = V[IDX(i, i)];
                        const double lim = fmax(TR_REL * fabs(th[i]), v > 0.0 && isfinite(v) ? TR_SIG * sqrt(v) : 0.0);
                        if (lim > 0.0) amax = fmin(amax, lim / fabs(d[i]));
                    }
                for (int k = 0; k < NLS; ++k) {
                    const double a = amax * ldexp(1.0, -k);
                    double* tk = slot_t(k);
                    for (int i = 0; i < Pt; ++i) tk[i] = fr[i] ? fmin(fmax(th[i] + a * d[i], lo[i]), hi[i]) : th[i];
                    F.skip[s0 + k] = 0;
                }
                for (int k = NLS; k < S; ++k) F.skip[s0 + k] = 1;
                c.evals += NLS;
            }
        }
    }
    if (to_hess) {
        int a = 0;
        for (int j = 0; j < Pt; ++j) {
            if (!fr[j]) continue;
            double h = c.hrel * fmax(fabs(th[j]), 1e-3);
            const double hjj = H[IDX(j, j)];
            if (c.hsig > 0.0 && isfinite(c.edm0) && hjj > 0.0 && isfinite(hjj))
                h = fmin(c.hsig / sqrt(hjj), 0.5 * fmax(fabs(th[j]), 1e-3));
            double* tp = slot_t(NLS + 2 * a);
            double* tm = slot_t(NLS + 2 * a + 1);
            for (int i = 0; i < Pt; ++i) { tp[i] = th[i]; tm[i] = th[i]; }
            tp[j] = fmin(th[j] + h, hi[j]);
            tm[j] = fmax(th[j] - h, lo[j]);
            F.skip[s0 + NLS + 2 * a] = 0;
            F.skip[s0 + NLS + 2 * a + 1] = 0;
            ++a;
        }
        for (int k = 0; k < NLS; ++k) F.skip[s0 + k] = 1;
        for (int k = NLS + 2 * a; k < S; ++k) F.skip[s0 + k] = 1;
        c.evals += 2 * a;
        c.phase = a > 0 ? PH_HESS : PH_DONE;
        if (a == 0) { c.status = BX_OK; c.edm = 0.0; }
    }
    if (c.phase != PH_DONE && c.evals >= c.max_evals) { c.phase = PH_DONE; c.status = BX_ENOTCONV; }
    if (c.phase == PH_DONE) for (int k = 0; k < S; ++k) F.skip[s0 + k] = 1;
    else atomicAdd(F.active, 1);
    F.ctl[jf] = c;
}

}  // namespace

struct FitState {
    int cap_fits = 0, P = 0, S = 0;
    FitDev dev{};
    int* active_h = nullptr;   // pinned
    cudaStream_t fs = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_n = -1, graph_ipl = -1;
    std::vector<void*> allocs;
};

void bx_fit_free(bx_model* m) {
    if (!m || !m->fit) return;
    FitState* s = m->fit;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->fs) cudaStreamDestroy(s->fs);
    if (s->active_h) cudaFreeHost(s->active_h);
    for (void* p : s->allocs) cudaFree(p);
    delete s;
    m->fit = nullptr;
}

#define CUF(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return bx_set_error(BX_ECUDA, "bx_fit: %s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static int fit_alloc(bx_model* m) {
    if (m->fit) return BX_OK;
    FitState* s = new FitState();
    m->fit = s;
    s->P = m->P;
    s->S = NLS + 2 * m->P;
    s->cap_fits = m->cap / s->S;
    const size_t n = s->cap_fits, P = s->P, ns = n * s->S;
    FitDev& D = s->dev;
    struct A { void** p; size_t bytes; } plan[] = {
        {(void**)&D.theta, n * P * 8}, {(void**)&D.g, n * P * 8},      {(void**)&D.f, n * 8},
        {(void**)&D.H, n * P * P * 8}, {(void**)&D.V, n * P * P * 8},  {(void**)&D.d, n * P * 8},
        {(void**)&D.lo, n * P * 8},    {(void**)&D.hi, n * P * 8},     {(void**)&D.fr, n * P},
        {(void**)&D.tt, ns * P * 8},   {(void**)&D.ft, ns * 8},        {(void**)&D.gt, ns * P * 8},
        {(void**)&D.skip, ns},         {(void**)&D.ctl, n * sizeof(FitCtl)}, {(void**)&D.active, 16},
        {(void**)&D.Pf, n * sizeof(int)},     {(void**)&D.Kf, n * sizeof(int)},
    };
    for (auto& a : plan) {
        CUF(cudaMalloc(a.p, a.bytes));
        s->allocs.push_back(*a.p);
    }
    CUF(cudaHostAlloc((void**)&s->active_h, sizeof(int), cudaHostAllocDefault));
    CUF(cudaStreamCreateWithFlags(&s->fs, cudaStreamNonBlocking));
    D.P = s->P;
    D.S = s->S;
    return BX_OK;
}

// Capture `ipl` iterations (evaluation of every slot in use + k_fit) into a graph.
static int fit_capture(bx_model* m, int n, int ipl) {
    FitState* s = m->fit;
    if (s->graph && s->graph_n == n && s->graph_ipl == ipl) return BX_OK;
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    cudaStream_t saved = m->stream;
    const int prof = m->prof_on;
    const unsigned char* saved_skip = m->w.skip;
    m->prof_on = 0;
    m->stream = s->fs;
    m->w.skip = s->dev.skip;
    FitDev D = s->dev;
    D.n = n;
    const int items = n * s->S;
    cudaGraph_t g = nullptr;
    int st = BX_OK;
    cudaError_t e = cudaStreamBeginCapture(s->fs, cudaStreamCaptureModeRelaxed);
    for (int it = 0; it < ipl && e == cudaSuccess && st == BX_OK; ++it) {
        if (it == ipl - 1) e = cudaMemsetAsync(D.active, 0, sizeof(int), s->fs);
        if (e != cudaSuccess) break;
        st = bx_enqueue_eval(m, items, D.tt, s->P, 1, 0, D.ft, D.gt);
        if (st) break;
        k_fit<<<(n + 63) / 64, 64, 0, s->fs>>>(D);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(s->fs, &g);
    m->stream = saved;
    m->prof_on = prof;
    m->w.skip = saved_skip;
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "bx_fit: graph capture: %s", cudaGetErrorString(e));
    s->graph_n = n;
    s->graph_ipl = ipl;
    return BX_OK;
}

extern "C" int bx_fit(bx_model* m, int n, const int* toy_idx, const double* theta0, const bx_fit_opts* opts,
                      double* theta_out, bx_fit_result* res) {
    if (!m || !theta0 || !theta_out || !res) return bx_set_error(BX_EINVAL, "bx_fit: NULL argument");
    BxRange range("bx_fit");
    bx_fit_opts o{};
    if (opts) o = *opts;
    if (o.tol_edm == 0.0) o.tol_edm = 1e-8;
    if (o.max_iter == 0) o.max_iter = 5000;
    if (o.iters_per_launch == 0) o.iters_per_launch = 4;
    if (!(o.tol_edm > 0.0) || o.max_iter < 1 || o.iters_per_launch < 1 || o.iters_per_launch > 256)
        return bx_set_error(BX_EINVAL, "bx_fit: invalid options");
    const int P = m->P, S = NLS + 2 * P, Kmax = m->Kmax;
    if (n < 1 || (long long)n * S > m->cap)
        return bx_set_error(BX_EINVAL, "bx_fit: %d fits need max_batch >= %lld (%d evaluation slots per fit)", n,
                            (long long)n * S, S);
    for (int j = 0; j < n; ++j)
        if (toy_idx && (toy_idx[j] < 0 || toy_idx[j] >= m->n_data))
            return bx_set_error(BX_EINVAL, "bx_fit: toy_idx[%d] out of range", j);
    std::vector<int> slot_toy((size_t)n * S);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < S; ++k) slot_toy[(size_t)j * S + k] = toy_idx ? toy_idx[j] : 0;
    int st = bx_set_items(m, n * S, slot_toy.data());
    if (st) return st;
    if ((st = fit_alloc(m))) return st;
    FitState* s = m->fit;
    // per-fit bounds and free flags in each fit's own layout
    std::vector<double> lo((size_t)n * P, -INFINITY), hi((size_t)n * P, INFINITY), th((size_t)n * S * P, 0.0);
    std::vector<unsigned char> fr((size_t)n * P, 0), skip((size_t)n * S, 1);
    std::vector<FitCtl> ctl(n);
    std::vector<int> Pf(n), Kf(n);
    const double hrel = m->precision == BX_FP64 ? 1e-3 : 1e-2;   // FD step of the Hessian
    for (int j = 0; j < n; ++j) {
        const int t = toy_idx ? toy_idx[j] : 0;
        const Toy& T = m->toys_h[(size_t)t * m->n_est];   // estimator 0 of the dataset
        Pf[j] = bx_public_P(m, t);
        Kf[j] = T.K;
        for (int p = 0; p < Pf[j]; ++p) {
            const int q = p < T.K ? p : Kmax + (p - T.K);   // slot in the Kmax layout of the options
            double l, h;
            unsigned char f;
            static const double dl[7] = {50.0, 0.0, 0.0, 1e-3, 0.0, 0.0, 0.05};
            static const double dh[7] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, 1.0, INFINITY};
            if (p < T.K) { l = 0.0; h = INFINITY; f = 1; }
            else if (p < T.K + 7) {
                l = dl[p - T.K];
                h = dh[p - T.K];
                f = (p - T.K == 6) ? (T.n_rad > 0 || T.n_r2 > 0) : 1;
            } else {   // LY, a, b, c of a further energy estimator
                l = dl[(p - T.K - 7) % 4];
                h = dh[(p - T.K - 7) % 4];
                f = 1;
            }
            if (o.lo) l = o.lo[q];
            if (o.hi) h = o.hi[q];
            if (o.free_mask) f = o.free_mask[q] ? 1 : 0;
            const double x = theta0[(size_t)j * P + p];
            if (!std::isfinite(x) || !(l <= h))
                return bx_set_error(BX_EINVAL, "bx_fit: theta0[%d][%d] or its bounds invalid", j, p);
            lo[(size_t)j * P + p] = l;
            hi[(size_t)j * P + p] = h;
            fr[(size_t)j * P + p] = f;
            th[(size_t)j * S * P + p] = std::min(std::max(x, l), h);   // slot 0: the start
        }
        skip[(size_t)j * S] = 0;
        const bool f64 = m->precision == BX_FP64;
        ctl[j] = FitCtl{PH_START, 0, 1, BX_ENOTCONV, o.max_iter, 0, 0, INFINITY, INFINITY,
                        f64 ? o.tol_edm : std::max(o.tol_edm, EDM_FLOOR_FP32), 0.0, 0.0, hrel,
                        f64 ? MU_CONV_FP64 : MU_CONV_FP32, f64 ? 0.0 : HSIG_FP32, 0.0};
    }
    FitDev& D = s->dev;
    CUF(cudaStreamSynchronize(m->stream));   // slot composition uploaded on the model stream
    CUF(cudaMemcpyAsync(D.tt, th.data(), th.size() * 8, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync(D.lo, lo.data(), lo.size() * 8, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync(D.hi, hi.data(), hi.size() * 8, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync(D.fr, fr.data(), fr.size(), cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync(D.skip, skip.data(), skip.size(), cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync(D.ctl, ctl.data(), ctl.size() * sizeof(FitCtl), cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.Pf, Pf.data(), Pf.size() * sizeof(int), cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.Kf, Kf.data(), Kf.size() * sizeof(int), cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemsetAsync(D.H, 0, (size_t)n * P * P * 8, s->fs));
    CUF(cudaStreamSynchronize(s->fs));
    if ((st = fit_capture(m, n, o.iters_per_launch))) return st;
    // a Newton iteration takes two evaluation rounds; the budget is in evaluation slots
    const int max_rounds = 2 * (o.max_iter / (2 * (P > 0 ? P : 1)) + 8) + 64;
    int rounds = 0;
    for (;;) {
        CUF(cudaGraphLaunch(s->graph, s->fs));
        CUF(cudaMemcpyAsync(s->active_h, D.active, sizeof(int), cudaMemcpyDeviceToHost, s->fs));
        CUF(cudaStreamSynchronize(s->fs));
        rounds += o.iters_per_launch;
        if (*s->active_h == 0 || rounds >= max_rounds) break;
    }
    unsigned err = 0;
    CUF(cudaMemcpy(&err, m->w.err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        CUF(cudaMemset(m->w.err, 0, sizeof(unsigned)));
        return bx_set_error(BX_ETIMEOUT, "bx_fit: a device-side wait exceeded its time budget");
    }
    std::vector<double> f(n);
    CUF(cudaMemcpy(theta_out, D.theta, (size_t)n * P * 8, cudaMemcpyDeviceToHost));
    CUF(cudaMemcpy(f.data(), D.f, (size_t)n * 8, cudaMemcpyDeviceToHost));
    CUF(cudaMemcpy(ctl.data(), D.ctl, ctl.size() * sizeof(FitCtl), cudaMemcpyDeviceToHost));
    int worst = BX_OK;
    for (int j = 0; j < n; ++j) {
        res[j].nll = f[j];
        res[j].edm = ctl[j].edm;
        res[j].iters = ctl[j].iters;
        res[j].n_evals = ctl[j].evals;
        res[j].status = ctl[j].phase == PH_DONE ? ctl[j].status : BX_ENOTCONV;
        res[j].n_at_bound = ctl[j].n_bound;
        res[j].damping = ctl[j].mu_fresh;
        if (res[j].status != BX_OK && worst == BX_OK) worst = res[j].status;
    }
    if (o.cov_out) CUF(cudaMemcpy(o.cov_out, D.V, (size_t)n * P * P * 8, cudaMemcpyDeviceToHost));
    if (worst != BX_OK) bx_set_error(worst, "bx_fit: not every fit converged (see the per-fit status)");
    return worst;
}
