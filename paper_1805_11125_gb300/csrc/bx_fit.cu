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
//          launch; of the steps satisfying the Armijo condition the one with the lowest -lnL is
//          accepted (below the FP32 noise floor of -lnL an undamped full step is accepted as
//          is) and HESS follows; if none qualifies the damping is raised and LS repeats (a
//          damping runaway retakes the Hessian with larger steps, at most MAX_RESTARTS times);
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
// The noise of a large toy's FP32 -lnL is above EDM_NOISE (it grows with the counts): each
// Hessian of an FP32 fit also estimates it, as the median over the parameters of
// |f(theta + h e_j) + f(theta - h e_j) - 2 f(theta) - H_jj h^2| / 2 (the second difference of f
// against the curvature from the gradients; their difference is rounding, the h^4 term being
// far smaller at steps of a conditional deviation).  An FP32 fit whose fresh, lightly damped
// step predicts less than FNOISE_K times that has reached its noise floor and is converged.
constexpr double FNOISE_K = 2.0;
// Largest fresh EDM at which an FP32 fit whose line search finds no decrease is taken to be at
// its noise floor (retaken Hessians, then BX_OK): within sqrt(2 x 1e-3) = 0.045 sigma.
constexpr double EDM_STALL = 1e-3;
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
constexpr double HSIG_FP32 = 1.0, HSIG_MAX = 64.0;
// A fit still running after every WIDEN_ITERS accepted steps doubles its finite-difference step
// (FP64: hrel up to HREL_MAX).  Such fits creep along long curved valleys of the nearly
// degenerate response parameters, where the curvature over one conditional deviation misleads
// the Newton step more than the curvature over a wider one.  On the 4096 toys of the batched-toy
// recipe: 3970 FP32 fits converged without it, 4000 with a doubling every 25 steps (every 10,
// 15, 35 or 50 steps, or a quadrupling every 25: 3974-3992; a starting step of 2 deviations:
// 3966).
constexpr int WIDEN_ITERS = 25;
constexpr double HREL_MAX = 16e-3;

// Trust region of the response, pile-up and radial parameters.  Far from the optimum the Newton
// step of these nearly degenerate parameters can be many times their value (the light yield,
// the resolution terms and kB trade off against each other), and a line search along it may
// accept a point from which the fit runs onto the bounds: a 5%-off start of the small joint
// model walked the resolution term b to 25 times its value with four parameters held at bounds.
// Near the optimum every step is well inside the region (a few standard deviations at most).
constexpr double TR_REL = 1.0, TR_SIG = 3.0;

// Hessians a fit may retake after a damping runaway before it gives up (BX_ENOTCONV).  Over the
// 4096 toys of the batched-toy recipe, 3 restarts raised the converged FP32 fits from 3919 to 3970
// (the other fits of the test suite unchanged or faster).
constexpr int MAX_RESTARTS = 3;

struct FitCtl {
    int phase, iters, evals, status, max_evals, fails, n_bound;
    double edm, edm0, tol, mu_min, mu_used, hrel, mu_conv, hsig, mu_fresh;
    double fnoise;   // FP32: rounding noise of -lnL estimated at the last Hessian (0 until then)
    int restarts;    // Hessians retaken after a damping runaway
};

struct FitDev {
    int n, P, S;
    int* Pf;                // per fit: parameters of its dataset's row (K_t + 7 + 4 (E - 1))
    int* Kf;                // per fit: rates (K_t), the parameters before the trust-region ones
    double *theta, *g, *f;  // accepted state per fit
    double *H, *V, *d;      // per fit
    double *lo, *hi;        // per fit
    unsigned char* fr;      // per fit
    double *tt, *ft, *gt;   // per slot: evaluation input and outputs
    unsigned char* skip;    // per slot
    FitCtl* ctl;
    int* active;
    // the work queue: run->n_fits fits wait, F.n slot blocks hold the fits in flight
    int E;                  // energy estimators per dataset (internal items per slot item)
    int* slot_fit;          // per slot block: the queued fit it holds, -1 idle
    int* next_fit;          // queue head
    const double *q_theta0, *q_lo, *q_hi;   // per queued fit [n_fits][P]
    const unsigned char* q_fr;              // [n_fits][P]
    const int *q_Pf, *q_Kf, *q_toy;         // [n_fits]
    const FitCtl* q_ctl0;                   // [n_fits]: initial state
    double *o_theta, *o_f;                  // results [n_fits][P], [n_fits]
    FitCtl* o_ctl;                          // [n_fits]
    int* toy_of;                            // the evaluation items' toys (internal items: slot item x E + e)
    // the persistent loop: rounds run, the loop's clock, the graph's loop handle
    int* rounds;
    unsigned long long* t0;
    int* timed_out;
    struct FitRun* run;                     // this call's parameters (read by the captured kernels)
    cudaGraphConditionalHandle handle;
};

// Parameters of one bx_fit call, in device memory so that one captured graph serves every call.
struct FitRun {
    int n_fits;                 // fits in the queue
    int max_rounds;             // evaluation-round budget of the batch
    unsigned long long budget_ns;   // device-clock budget of the batch
    double* o_V;                // [n_fits][P][P] covariance out, or nullptr
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

// Put queued fit qf into slot block jf: its start in slot 0 (to be evaluated next round), its
// bounds, free flags and state, its dataset on the slot's evaluation items.
__device__ void slot_load(const FitDev& F, int jf, int qf) {
    const int P = F.P, S = F.S;
    const size_t s0 = (size_t)jf * S;
    F.slot_fit[jf] = qf;
    for (int i = 0; i < P; ++i) {
        F.tt[s0 * P + i] = F.q_theta0[(size_t)qf * P + i];
        F.lo[(size_t)jf * P + i] = F.q_lo[(size_t)qf * P + i];
        F.hi[(size_t)jf * P + i] = F.q_hi[(size_t)qf * P + i];
        F.fr[(size_t)jf * P + i] = F.q_fr[(size_t)qf * P + i];
    }
    for (int i = 0; i < P * P; ++i) F.H[(size_t)jf * P * P + i] = 0.0;
    F.Pf[jf] = F.q_Pf[qf];
    F.Kf[jf] = F.q_Kf[qf];
    F.ctl[jf] = F.q_ctl0[qf];
    const int toy = F.q_toy[qf];
    for (int k = 0; k < S; ++k) {
        F.skip[s0 + k] = k == 0 ? 0 : 1;
        for (int e = 0; e < F.E; ++e) F.toy_of[(s0 + k) * F.E + e] = toy * F.E + e;
    }
}

// A finished fit's result leaves its slot block: theta (its start beyond the fit's own P, where
// the slot may hold a longer fit's values) and, when asked for, the covariance.
__device__ void slot_store(const FitDev& F, int jf, const FitCtl& c) {
    const int P = F.P, qf = F.slot_fit[jf], Pt = F.Pf[jf];
    for (int i = 0; i < P; ++i)
        F.o_theta[(size_t)qf * P + i] = i < Pt ? F.theta[(size_t)jf * P + i] : F.q_theta0[(size_t)qf * P + i];
    F.o_f[qf] = F.f[jf];
    F.o_ctl[qf] = c;
    double* oV = F.run->o_V;
    if (oV) {
        const double* V = F.V + (size_t)jf * P * P;
        for (int i = 0; i < P; ++i)
            for (int j = 0; j < P; ++j) oV[(size_t)qf * P * P + IDX(i, j)] = (i < Pt && j < Pt) ? V[IDX(i, j)] : 0.0;
    }
}

// Fill every slot block from the queue (before the first round).
__global__ void k_fit_init(FitDev F) {
    const int jf = blockIdx.x * blockDim.x + threadIdx.x;
    if (jf >= F.n) return;
    const int qf = atomicAdd(F.next_fit, 1);
    if (qf < F.run->n_fits) {
        slot_load(F, jf, qf);
    } else {
        F.slot_fit[jf] = -1;
        for (int k = 0; k < F.S; ++k) F.skip[(size_t)jf * F.S + k] = 1;
    }
}

// For the autotuner: every slot of a block evaluates the block's start point (a full round).
__global__ void k_fit_tune_fill(FitDev F) {
    const int jf = blockIdx.x, k = threadIdx.x;   // block = slot block, thread = slot
    if (jf >= F.n || k >= F.S || F.slot_fit[jf] < 0) return;
    const size_t s0 = (size_t)jf * F.S;
    for (int i = 0; i < F.P; ++i) F.tt[(s0 + k) * F.P + i] = F.tt[s0 * F.P + i];
    F.skip[s0 + k] = 0;
}

// The loop's clock starts with its first round.
__global__ void k_fit_clock(FitDev F) {
    if (*F.t0 == 0ull) *F.t0 = globaltimer();
}

// End of a loop body: continue while a fit is active, within the round and time budgets.
__global__ void k_fit_ctl(FitDev F) {
    const int r = ++*F.rounds;
    const bool more = *F.active > 0 && r < F.run->max_rounds;
    const bool late = globaltimer() - *F.t0 > F.run->budget_ns;
    if (more && late) *F.timed_out = 1;
    cudaGraphSetConditional(F.handle, more && !late ? 1u : 0u);
}

__global__ void k_fit(FitDev F) {
    const int jf = blockIdx.x * blockDim.x + threadIdx.x;
    if (jf >= F.n || F.slot_fit[jf] < 0) return;
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
        // column j: the central difference of the gradients at theta +- h e_j; where one side was
        // not evaluable (outside the model's domain, or h below the resolution of theta_j) the
        // one-sided difference with the accepted point; with neither, no curvature (damping
        // then carries that direction)
        auto finite_at = [&](int k) {
            if (!isfinite(F.ft[s0 + k])) return false;
            const double* gk = slot_g(k);
            for (int i = 0; i < Pt; ++i)
                if (!isfinite(gk[i])) return false;
            return true;
        };
        int a = 0, ne = 0;
        double res[PFMAX];
        for (int j = 0; j < Pt; ++j) {
            if (!fr[j]) continue;
            const int kp = NLS + 2 * a, km = kp + 1;
            const double up = slot_t(kp)[j], dn = slot_t(km)[j];
            const bool okp = finite_at(kp) && up > th[j], okm = finite_at(km) && dn < th[j];
            const double* ga = okp ? slot_g(kp) : g;
            const double* gb = okm ? slot_g(km) : g;
            const double du = (okp ? up : th[j]) - (okm ? dn : th[j]);
            for (int i = 0; i < Pt; ++i) H[IDX(i, j)] = (fr[i] && du > 0.0) ? (ga[i] - gb[i]) / du : 0.0;
            if (c.hsig > 0.0 && okp && okm && up - th[j] == th[j] - dn) {   // symmetric: f's noise
                const double h = up - th[j];
                res[ne++] = 0.5 * fabs(F.ft[s0 + kp] + F.ft[s0 + km] - 2.0 * F.f[jf] - H[IDX(j, j)] * h * h);
            }
            ++a;
        }
        if (ne > 0) {   // median (insertion sort of at most PFMAX values)
            for (int i = 1; i < ne; ++i)
                for (int k = i; k > 0 && res[k - 1] > res[k]; --k) {
                    const double t = res[k];
                    res[k] = res[k - 1];
                    res[k - 1] = t;
                }
            c.fnoise = ne & 1 ? res[ne / 2] : 0.5 * (res[ne / 2 - 1] + res[ne / 2]);
        }
        newdir = fresh = true;
    } else if (c.phase == PH_LS) {
        // the NLS step lengths were evaluated together: of those with sufficient decrease
        // (Armijo), the one with the lowest -lnL -- not the longest, which in a curved valley
        // (the correlated resolution terms) can land far out on a descent that a shorter step
        // beats.  At the noise floor of the FP32 -lnL (an undamped step predicting less than
        // EDM_NOISE) the full step counts as a decrease while it stays within the noise.
        int acc = -1;
        double fbest = 0.0;
        for (int k = 0; k < NLS; ++k) {
            const double fk = F.ft[s0 + k];
            if (!isfinite(fk)) continue;
            double gs = 0.0;
            const double* tk = slot_t(k);
            for (int i = 0; i < Pt; ++i) gs += g[i] * (tk[i] - th[i]);
            const double nz = fmax(EDM_NOISE, c.fnoise);
            const bool noise_floor = k == 0 && c.mu_used <= c.mu_conv && c.edm0 < nz && fk <= F.f[jf] + 2.0 * nz;
            if ((fk <= F.f[jf] + 1e-4 * gs || noise_floor) && (acc < 0 || fk < fbest)) {
                acc = k;
                fbest = fk;
            }
        }
        if (acc >= 0) {
            for (int i = 0; i < Pt; ++i) { th[i] = slot_t(acc)[i]; g[i] = slot_g(acc)[i]; }
            F.f[jf] = F.ft[s0 + acc];
            c.iters++;
            c.mu_min = 0.0;
            to_hess = true;
            if (c.iters % WIDEN_ITERS == 0) {   // a long fit: wider finite-difference steps
                if (c.hsig > 0.0) c.hsig = fmin(2.0 * c.hsig, HSIG_MAX);
                else c.hrel = fmin(2.0 * c.hrel, HREL_MAX);
            }
        } else if (c.hsig > 0.0 && c.edm0 < fmax(c.tol, EDM_STALL)) {
            // an FP32 fit whose fresh step predicts little (or whose Hessian is indefinite) and
            // no trial lowers -lnL: the curvature of a weak direction is lost in the gradients'
            // rounding noise over a step of HSIG conditional deviations, so the Hessian is taken
            // again with 4x the step; once that reaches HSIG_MAX the point is the optimum to
            // within the FP32 noise floor (an FP64 polish resolves the rest)
            c.fails++;
            if (c.hsig < HSIG_MAX) {
                c.hsig *= 4.0;
                to_hess = true;
            } else {
                c.phase = PH_DONE;
                c.status = BX_OK;
            }
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
        if (mu < 0.0 && c.restarts < MAX_RESTARTS) {
            // damping runaway (no damping up to 1e8 gave a positive definite matrix, or line
            // searches failed at every damping): the Hessian is taken again with 4x the step,
            // as MIGRAD falls back to a fresh second-derivative matrix when its update fails
            c.restarts++;
            c.mu_min = 0.0;
            if (c.hsig > 0.0) c.hsig = fmin(4.0 * c.hsig, HSIG_MAX);
            else c.hrel *= 4.0;
            to_hess = true;
        } else if (mu < 0.0) {
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
            if (fresh && c.edm < fmax(c.tol, FNOISE_K * c.fnoise) && mu <= c.mu_conv) {
                c.phase = PH_DONE;
                c.status = BX_OK;
            } else {
                c.phase = PH_LS;
                // trust region of the response, pile-up and radial parameters (everything after the
                // rates), per parameter: a trial step moves none of them by more than TR_REL of its
                // magnitude or TR_SIG of its standard deviation under the current Hessian, whichever
                // is larger.  A component beyond its limit is clipped and the others keep their
                // length (scaling the whole step instead let one tightly limited parameter stall
                // every other one, and a first step from 10% out had sent the constant noise term c
                // to hundreds of times its optimum).
                double lim[PFMAX];
                for (int i = 0; i < Pt; ++i) {
                    lim[i] = INFINITY;
                    if (i >= Kt && act[i]) {
                        const double v = V[IDX(i, i)];
                        const double l = fmax(TR_REL * fabs(th[i]), v > 0.0 && isfinite(v) ? TR_SIG * sqrt(v) : 0.0);
                        if (l > 0.0) lim[i] = l;
                    }
                }
                for (int k = 0; k < NLS; ++k) {
                    const double a = ldexp(1.0, -k);
                    double* tk = slot_t(k);
                    for (int i = 0; i < Pt; ++i)
                        tk[i] = fr[i] ? fmin(fmax(th[i] + fmin(fmax(a * d[i], -lim[i]), lim[i]), lo[i]), hi[i]) : th[i];
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
    if (c.phase == PH_DONE) {   // result out, the next queued fit in
        slot_store(F, jf, c);
        const int qf = atomicAdd(F.next_fit, 1);
        if (qf < F.run->n_fits) {
            slot_load(F, jf, qf);
            atomicAdd(F.active, 1);
        } else {
            F.slot_fit[jf] = -1;
            for (int k = 0; k < S; ++k) F.skip[s0 + k] = 1;
        }
        return;
    }
    atomicAdd(F.active, 1);
    F.ctl[jf] = c;
}

}  // namespace

struct FitState {
    int cap_fits = 0, P = 0, S = 0;
    FitDev dev{};
    cudaStream_t fs = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_F = -1, graph_ipl = -1;
    cudaGraphConditionalHandle handle = 0;
    size_t q_cap = 0, v_cap = 0;             // queued fits the queue buffers hold (v: with covariance)
    double* o_V = nullptr;                   // covariance out [v_cap][P][P]
    std::vector<void*> allocs, q_allocs;
    int tuned_F = 0, tuned_tile = -1;        // wave shape and forward tile chosen by the autotuner
    double tuned_evals_per_s = 0.0;
    bx_fit_plan plan{};
};

void bx_fit_free(bx_model* m) {
    if (!m || !m->fit) return;
    FitState* s = m->fit;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->fs) cudaStreamDestroy(s->fs);
    for (void* p : s->allocs) cudaFree(p);
    for (void* p : s->q_allocs) cudaFree(p);
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
        {(void**)&D.slot_fit, n * sizeof(int)}, {(void**)&D.next_fit, 16}, {(void**)&D.rounds, 16},
        {(void**)&D.t0, 16}, {(void**)&D.timed_out, 16}, {(void**)&D.run, sizeof(FitRun)},
    };
    for (auto& a : plan) {
        CUF(cudaMalloc(a.p, a.bytes));
        s->allocs.push_back(*a.p);
    }
    CUF(cudaStreamCreateWithFlags(&s->fs, cudaStreamNonBlocking));
    D.P = s->P;
    D.S = s->S;
    D.E = m->n_est;
    D.toy_of = const_cast<int*>(m->w.toy_of);
    return BX_OK;
}

// Queue buffers for n fits (grown on demand; a new set of pointers invalidates the graph).
static int queue_alloc(bx_model* m, size_t n, bool cov) {
    FitState* s = m->fit;
    if (n <= s->q_cap && (!cov || n <= s->v_cap)) return BX_OK;
    for (void* p : s->q_allocs) cudaFree(p);
    s->q_allocs.clear();
    const size_t P = s->P, cap = std::max(n, s->q_cap);
    FitDev& D = s->dev;
    struct A { void** p; size_t bytes; } plan[] = {
        {(void**)&D.q_theta0, cap * P * 8}, {(void**)&D.q_lo, cap * P * 8}, {(void**)&D.q_hi, cap * P * 8},
        {(void**)&D.q_fr, cap * P},         {(void**)&D.q_Pf, cap * 4},     {(void**)&D.q_Kf, cap * 4},
        {(void**)&D.q_toy, cap * 4},        {(void**)&D.q_ctl0, cap * sizeof(FitCtl)},
        {(void**)&D.o_theta, cap * P * 8},  {(void**)&D.o_f, cap * 8},      {(void**)&D.o_ctl, cap * sizeof(FitCtl)},
        {(void**)&s->o_V, cov ? cap * P * P * 8 : 16},
    };
    for (auto& a : plan) {
        CUF(cudaMalloc(a.p, a.bytes));
        s->q_allocs.push_back(*a.p);
    }
    s->q_cap = cap;
    s->v_cap = cov ? cap : 0;
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    return BX_OK;
}

// The persistent batch: one graph whose conditional while node repeats the body
//   k_fit_clock, ipl x {evaluate the F slot blocks (F S items), k_fit}, k_fit_ctl
// until k_fit_ctl clears the loop condition (no fit active, or a budget spent); the active count
// is cleared before the body's last k_fit, which counts the fits still running.
static int fit_capture(bx_model* m, int F, int ipl) {
    FitState* s = m->fit;
    if (s->graph && s->graph_F == F && s->graph_ipl == ipl) return BX_OK;
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CUF(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    cudaGraphNode_t node;
    cudaGraphNodeParams cp{};
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return bx_set_error(BX_ECUDA, "bx_fit: conditional graph node: %s", cudaGetErrorString(e));
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    FitDev D = s->dev;
    D.n = F;
    D.handle = h;
    s->dev.handle = h;
    cudaStream_t saved = m->stream;
    const int prof = m->prof_on;
    const unsigned char* saved_skip = m->w.skip;
    m->prof_on = 0;
    m->stream = s->fs;
    m->w.skip = s->dev.skip;
    int st = BX_OK;
    e = cudaStreamBeginCaptureToGraph(s->fs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        k_fit_clock<<<1, 1, 0, s->fs>>>(D);
        e = cudaGetLastError();
    }
    for (int it = 0; it < ipl && e == cudaSuccess && st == BX_OK; ++it) {
        if (it == ipl - 1) e = cudaMemsetAsync(D.active, 0, sizeof(int), s->fs);
        if (e != cudaSuccess) break;
        st = bx_enqueue_eval(m, F * s->S, D.tt, s->P, 1, 0, D.ft, D.gt);
        if (st) break;
        k_fit<<<(F + 63) / 64, 64, 0, s->fs>>>(D);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && st == BX_OK) {
        k_fit_ctl<<<1, 1, 0, s->fs>>>(D);
        e = cudaGetLastError();
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s->fs, &captured);
    m->stream = saved;
    m->prof_on = prof;
    m->w.skip = saved_skip;
    if (st) {
        cudaGraphDestroy(g);
        return st;
    }
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "bx_fit: graph capture: %s", cudaGetErrorString(e));
    s->graph_F = F;
    s->graph_ipl = ipl;
    return BX_OK;
}

// The autotuner: with the slot blocks loaded (k_fit_init), time one evaluation round of the
// first F blocks for F = the largest whole multiple of the GPU's SM count in evaluation items
// and its halves, and each forward tile shape of the model; keep the fastest tile shape and the
// smallest F within 10% of the best throughput (fewer fits in flight: shorter rounds for the
// last fits of the queue).  Returns the chosen F.
static int fit_autotune(bx_model* m, int Fmax) {
    FitState* s = m->fit;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<int> cand;
    for (int F = Fmax; F >= 1 && (int)cand.size() < 5; F /= 2) cand.push_back(F);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return Fmax;
    cudaStream_t saved = m->stream;
    const unsigned char* saved_skip = m->w.skip;
    m->stream = s->fs;
    m->w.skip = s->dev.skip;
    const int n_tiles = bx_fwd_tile_variants(m);
    double best = 0.0;
    int best_tile = 0;
    std::vector<double> thr(cand.size(), 0.0);
    for (int tv = 0; tv < n_tiles; ++tv) {
        bx_set_fwd_tile(m, tv);
        for (size_t c = 0; c < cand.size(); ++c) {
            const int items = cand[c] * s->S;
            float ms = 0.f, t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {   // first call warms up
                cudaEventRecord(a, s->fs);
                bx_enqueue_eval(m, items, s->dev.tt, s->P, 1, 0, s->dev.ft, s->dev.gt);
                cudaEventRecord(b, s->fs);
                cudaEventSynchronize(b);
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) t = std::min(t, ms);
            }
            const double v = items / (t / 1e3);
            if (v > best) { best = v; best_tile = tv; }
            if (tv == 0 || v > thr[c]) thr[c] = v;
        }
    }
    bx_set_fwd_tile(m, best_tile);
    m->stream = saved;
    m->w.skip = saved_skip;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    // the largest wave within 10% of the best rate: the timed rounds have every slot busy, while
    // a fit's rounds in flight use a third of its slots on average (8 trials or 2 P Hessian
    // points of 8 + 2 P), so a wave that only just fills the GPU here starves it in the loop
    // (4096 toys: 256 in flight ran at 226k evaluations/s against 447k with all of them)
    int F = cand.back();
    const double top = *std::max_element(thr.begin(), thr.end());
    for (size_t c = cand.size(); c-- > 0;)
        if (thr[c] >= 0.9 * top) F = cand[c];   // candidates descend: the last one found is the largest
    s->tuned_F = F;
    s->tuned_tile = best_tile;
    s->tuned_evals_per_s = best;
    (void)sms;
    return F;
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
    if (o.time_budget_s == 0.0) o.time_budget_s = 300.0;
    if (!(o.tol_edm > 0.0) || o.max_iter < 1 || o.iters_per_launch < 1 || o.iters_per_launch > 256 ||
        !(o.time_budget_s > 0.0) || o.fits_in_flight < 0)
        return bx_set_error(BX_EINVAL, "bx_fit: invalid options");
    const int P = m->P, S = NLS + 2 * P, Kmax = m->Kmax;
    if (n < 1) return bx_set_error(BX_EINVAL, "bx_fit: n = %d", n);
    if (m->cap < S) return bx_set_error(BX_EINVAL, "bx_fit: max_batch >= %d needed (%d evaluation slots per fit)", S, S);
    for (int j = 0; j < n; ++j)
        if (toy_idx && (toy_idx[j] < 0 || toy_idx[j] >= m->n_data))
            return bx_set_error(BX_EINVAL, "bx_fit: toy_idx[%d] out of range", j);
    int st;
    if ((st = fit_alloc(m))) return st;
    FitState* s = m->fit;
    if ((st = queue_alloc(m, (size_t)n, o.cov_out != nullptr))) return st;
    // per-fit start, bounds, free flags and state in each fit's own layout
    std::vector<double> lo((size_t)n * P, -INFINITY), hi((size_t)n * P, INFINITY), th((size_t)n * P, 0.0);
    std::vector<unsigned char> fr((size_t)n * P, 0);
    std::vector<FitCtl> ctl(n);
    std::vector<int> Pf(n), Kf(n), toy(n);
    const double hrel = m->precision == BX_FP64 ? 1e-3 : 1e-2;   // FD step of the Hessian
    const bool f64 = m->precision == BX_FP64;
    for (int j = 0; j < n; ++j) {
        const int t = toy_idx ? toy_idx[j] : 0;
        const Toy& T = m->toys_h[(size_t)t * m->n_est];   // estimator 0 of the dataset
        toy[j] = t;
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
            th[(size_t)j * P + p] = std::min(std::max(x, l), h);
        }
        ctl[j] = FitCtl{PH_START, 0, 1, BX_ENOTCONV, o.max_iter, 0, 0, INFINITY, INFINITY,
                        f64 ? o.tol_edm : std::max(o.tol_edm, EDM_FLOOR_FP32), 0.0, 0.0, hrel,
                        f64 ? MU_CONV_FP64 : MU_CONV_FP32, f64 ? 0.0 : HSIG_FP32, 0.0};
    }
    FitDev& D = s->dev;
    CUF(cudaStreamSynchronize(m->stream));   // nothing of the model stream still reads the items' toys
    CUF(cudaMemcpyAsync((void*)D.q_theta0, th.data(), th.size() * 8, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.q_lo, lo.data(), lo.size() * 8, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.q_hi, hi.data(), hi.size() * 8, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.q_fr, fr.data(), fr.size(), cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.q_Pf, Pf.data(), Pf.size() * 4, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.q_Kf, Kf.data(), Kf.size() * 4, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.q_toy, toy.data(), toy.size() * 4, cudaMemcpyHostToDevice, s->fs));
    CUF(cudaMemcpyAsync((void*)D.q_ctl0, ctl.data(), ctl.size() * sizeof(FitCtl), cudaMemcpyHostToDevice, s->fs));

    // fits in flight: the caller's choice, else the autotuner's (measured once per model and batch size)
    const int Fmax = std::min(s->cap_fits, n);
    int F = o.fits_in_flight > 0 ? std::min(o.fits_in_flight, Fmax) : 0;
    {   // n_fits for k_fit_init; the budgets follow once F is known
        FitRun pre{n, 0, 0ull, nullptr};
        CUF(cudaMemcpyAsync(D.run, &pre, sizeof pre, cudaMemcpyHostToDevice, s->fs));
    }
    auto load = [&](int nslots) -> int {
        D.n = nslots;
        CUF(cudaMemsetAsync(D.next_fit, 0, sizeof(int), s->fs));
        k_fit_init<<<(nslots + 63) / 64, 64, 0, s->fs>>>(D);
        CUF(cudaGetLastError());
        return BX_OK;
    };
    if (F == 0) {
        if (s->tuned_F > 0 && s->tuned_F <= Fmax && s->plan.fits == n) {
            F = s->tuned_F;
        } else {
            if ((st = load(Fmax))) return st;
            k_fit_tune_fill<<<Fmax, std::max(32, (S + 31) / 32 * 32), 0, s->fs>>>(D);
            CUF(cudaGetLastError());
            CUF(cudaStreamSynchronize(s->fs));
            F = fit_autotune(m, Fmax);
        }
    }
    if ((st = load(F))) return st;
    CUF(cudaMemsetAsync(D.rounds, 0, sizeof(int), s->fs));
    CUF(cudaMemsetAsync(D.t0, 0, sizeof(unsigned long long), s->fs));
    CUF(cudaMemsetAsync(D.timed_out, 0, sizeof(int), s->fs));
    // a Newton iteration takes two evaluation rounds; the budget is in evaluation slots, and the
    // queue adds the rounds of its later fits
    FitRun run{n, (2 * (o.max_iter / (2 * (P > 0 ? P : 1)) + 8) + 64) * ((n + F - 1) / F),
               (unsigned long long)(o.time_budget_s * 1e9), o.cov_out ? s->o_V : nullptr};
    CUF(cudaMemcpyAsync(D.run, &run, sizeof run, cudaMemcpyHostToDevice, s->fs));
    m->toy_cached.assign(m->toy_cached.size(), -1);   // the device now sets the items' toys
    if ((st = fit_capture(m, F, o.iters_per_launch))) return st;
    CUF(cudaGraphLaunch(s->graph, s->fs));
    CUF(cudaStreamSynchronize(s->fs));
    unsigned err = 0;
    CUF(cudaMemcpy(&err, m->w.err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        CUF(cudaMemset(m->w.err, 0, sizeof(unsigned)));
        return bx_set_error(BX_ETIMEOUT, "bx_fit: a device-side wait exceeded its time budget");
    }
    int rounds = 0, timed_out = 0, next = 0;
    std::vector<int> slot_fit(F);
    CUF(cudaMemcpy(&rounds, D.rounds, sizeof(int), cudaMemcpyDeviceToHost));
    CUF(cudaMemcpy(&timed_out, D.timed_out, sizeof(int), cudaMemcpyDeviceToHost));
    CUF(cudaMemcpy(&next, D.next_fit, sizeof(int), cudaMemcpyDeviceToHost));
    CUF(cudaMemcpy(slot_fit.data(), D.slot_fit, F * sizeof(int), cudaMemcpyDeviceToHost));
    // fits still in their slots when the loop stopped (a budget spent): their current state
    std::vector<double> f(n);
    std::vector<FitCtl> oc(n);
    CUF(cudaMemcpy(theta_out, D.o_theta, (size_t)n * P * 8, cudaMemcpyDeviceToHost));
    CUF(cudaMemcpy(f.data(), D.o_f, (size_t)n * 8, cudaMemcpyDeviceToHost));
    CUF(cudaMemcpy(oc.data(), D.o_ctl, (size_t)n * sizeof(FitCtl), cudaMemcpyDeviceToHost));
    std::vector<char> finished(n, 0), running(n, 0);
    for (int j = 0; j < std::min(next, n); ++j) finished[j] = 1;
    for (int jf = 0; jf < F; ++jf)
        if (slot_fit[jf] >= 0) {
            const int qf = slot_fit[jf];
            finished[qf] = 0;
            running[qf] = 1;
            CUF(cudaMemcpy(theta_out + (size_t)qf * P, D.theta + (size_t)jf * P, P * 8, cudaMemcpyDeviceToHost));
            CUF(cudaMemcpy(&f[qf], D.f + jf, 8, cudaMemcpyDeviceToHost));
            CUF(cudaMemcpy(&oc[qf], D.ctl + jf, sizeof(FitCtl), cudaMemcpyDeviceToHost));
        }
    int worst = BX_OK;
    for (int j = 0; j < n; ++j) {
        const bool started = finished[j] || running[j];
        if (!started) {   // never left the queue
            for (int p = 0; p < P; ++p) theta_out[(size_t)j * P + p] = th[(size_t)j * P + p];
            oc[j] = ctl[j];
            f[j] = INFINITY;
        }
        res[j].nll = f[j];
        res[j].edm = oc[j].edm;
        res[j].iters = oc[j].iters;
        res[j].n_evals = started ? oc[j].evals : 0;
        res[j].status = finished[j] && oc[j].phase == PH_DONE ? oc[j].status
                        : timed_out                           ? BX_ETIMEOUT
                                                              : BX_ENOTCONV;
        res[j].n_at_bound = oc[j].n_bound;
        res[j].damping = oc[j].mu_fresh;
        if (res[j].status != BX_OK && worst == BX_OK) worst = res[j].status;
    }
    if (o.cov_out) {
        CUF(cudaMemcpy(o.cov_out, s->o_V, (size_t)n * P * P * 8, cudaMemcpyDeviceToHost));
        for (int jf = 0; jf < F; ++jf)
            if (slot_fit[jf] >= 0)
                CUF(cudaMemcpy(o.cov_out + (size_t)slot_fit[jf] * P * P, D.V + (size_t)jf * P * P, (size_t)P * P * 8,
                               cudaMemcpyDeviceToHost));
    }
    s->plan = bx_fit_plan{n, F, S, o.iters_per_launch, 1, rounds, s->tuned_tile, s->tuned_evals_per_s};
    if (worst != BX_OK) bx_set_error(worst, "bx_fit: not every fit converged (see the per-fit status)");
    return worst;
}

extern "C" int bx_fit_last_plan(const bx_model* m, bx_fit_plan* out) {
    if (!m || !out) return bx_set_error(BX_EINVAL, "NULL argument");
    if (!m->fit) return bx_set_error(BX_EINVAL, "no fit has run on this model");
    *out = m->fit->plan;
    return BX_OK;
}
