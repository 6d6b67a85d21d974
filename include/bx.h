/*
 * bx.h -- C ABI of the GB300 (sm_103a) binned Poisson -lnL engine for the Borexino-style
 * multivariate spectral fit of arXiv:1805.11125.
 *
 * What one evaluation computes (Sec. 3 of the paper; readings where the paper is silent
 * are stated inline):
 *   Eq. 1  every species' true-energy shape s_k[i] is mapped to the observable (npe) by
 *          the response R[m,i]: Birks quenching Q_i = sum_{j<i} dE/(1+kB S_j) +
 *          dE/(2(1+kB S_i)) (S = caller-supplied stopping power), mean mu_i = LY Q_i,
 *          Gaussian resolution of variance a mu_i + b mu_i^2 + c, bin-integrated over
 *          [m w, (m+1) w) and normalised to the mass above 0 npe;
 *          v_k[m] = sum_i R[m,i] s_k[i].
 *   Eq. 3  two energy spectra, TFC-vetoed (weight 1 - t_k) and TFC-tagged (weight t_k),
 *          lambda_h[m] = sum_k r_k c_{h,k} v_k[m]; without tag fractions a single
 *          spectrum with weight 1.
 *   Eq. 2  pile-up with scale eps and random-trigger spectrum g (sum g = 1):
 *          mu_h[m] = (1-eps) lambda_h[m] + eps sum_{d=0}^{min(m,L-1)} g[d] lambda_h[m-d].
 *   Eq. 4  radial and pulse-shape histograms: window marginals of the TFC-vetoed species
 *          spectra after pile-up, times radial bin probabilities (internal: uniform in
 *          volume; external: exp(-(r_iv - r)/(att_len s_r)) r^2, in a sphere r_fid) and
 *          caller-supplied pulse-shape bin probabilities.
 *   -lnL  = sum over all bins of mu - n + n ln(n/mu)   (n ln(n/mu) := 0 at n = 0),
 *          the Baker-Cousins form: it differs from sum(mu - n ln mu + ln n!) by the
 *          data-only constant sum(n - n ln n + ln n!), so -2 lnL differences are equal.
 *
 * Parameter vector of a toy with K species (P = K + 7), FP64:
 *   theta = [r_0 .. r_{K-1}, LY, a, b, c, kB, eps, s_r]
 * r_k are expected event counts of species k (exposure folded in).
 *
 * Conventions for every call:
 *   - status codes never abort; bx_last_error() gives a thread-local message;
 *   - the caller owns every input array; bx_model_create copies them to the device;
 *   - the library owns all device buffers of a model until bx_model_destroy;
 *   - work runs on the CUDA stream given at creation (or bx_model_set_stream);
 *   - host-pointer calls return after their results are in host memory;
 *     device-pointer calls (device_ptrs = 1) return once the work is enqueued.
 */
#ifndef BX_H
#define BX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bx_model bx_model;                 /* opaque; owns device memory */

typedef enum {
    BX_OK = 0,
    BX_EINVAL = -1,     /* invalid argument or model description */
    BX_ENOMEM = -2,     /* device or host allocation failed */
    BX_ECUDA = -3,      /* a CUDA call failed (message in bx_last_error) */
    BX_EDOMAIN = -4,    /* expected count <= 0 in a bin with data, or sigma^2 <= 0: -lnL = +inf */
    BX_ETIMEOUT = -5,   /* a device-side wait ran out of its time budget */
    BX_ENOTCONV = -6    /* a fit did not converge within its iteration budget */
} bx_status;

typedef enum {
    BX_FP64 = 0,        /* every step in FP64 on the CUDA cores (reference GPU form) */
    BX_FP32 = 1,        /* mixed: response generated and contracted in FP32 on the CUDA cores
                           (round-to-nearest, compensated accumulation); FP64 column
                           normalisation, spectra assembly, -lnL sum and fit update */
    BX_BF16X3 = 2,      /* the 2D models (discrimination regime, joint grid): as BX_FP32, but
                           the response GEMM's operands are split in three BF16 parts (hi on
                           a grid fixed for the contraction, BF16 mid and lo; 6 of the 9
                           products) on tcgen05.mma kind::f16 with FP32 accumulation in tensor
                           memory, in place of the TF32 parts of BX_FP32 (~24 instead of ~30
                           significant bits per operand) */
    BX_TF32X3 = 3       /* the 1D models: as BX_FP32, but the species-resolved contraction
                           runs on the tensor cores with three-part TF32 operands (hi on a
                           per-row grid, TF32 mid and lo) and FP32 accumulation in tensor
                           memory; the 2D models always run their GEMMs on the tensor cores */
} bx_precision;

enum { BX_RAD_INTERNAL = 0, BX_RAD_EXTERNAL = 1 };

/* One dataset (toy) and its model.  All arrays are host FP64 (rad_class int32) and are
 * copied at creation. */
typedef struct {
    int n_grid;                 /* true-energy points N; E_i = (i + 1/2) e_max / N */
    double e_max;               /* MeV */
    int n_species;              /* K, 1..16 */
    const double* shapes;       /* [K][N], each row >= 0 (rows need not sum to 1) */
    const double* stop_pow;     /* [N] stopping power on the grid, MeV/cm (> 0) */
    const double* tag_frac;     /* [K] TFC tagging fraction t_k, or NULL: one spectrum */
    int n_pileup;               /* L, 1..4096 */
    const double* pileup;       /* [L] random-trigger spectrum in bins of `width` */
    double width;               /* npe per bin */
    int m_lo, m_hi;             /* energy window = bins [m_lo, m_hi) of the axis [0, m_hi) */
    const double* counts_sub;   /* [m_hi - m_lo] vetoed (or single) spectrum data */
    const double* counts_tag;   /* [m_hi - m_lo] tagged spectrum data (with tag_frac) */
    int n_rad;                  /* radial bins over [0, r_fid), 0 = no radial term */
    const int* rad_class;       /* [K] BX_RAD_INTERNAL / BX_RAD_EXTERNAL */
    double r_fid, r_iv, att_len;/* fiducial radius, vessel radius, attenuation length (m) */
    const double* counts_rad;   /* [n_rad] */
    int n_psd;                  /* pulse-shape bins, 0 = no pulse-shape term */
    const double* psd_prob;     /* [K][n_psd] bin probabilities of each species */
    const double* counts_psd;   /* [n_psd] */
    /* 2D histograms of the TFC-vetoed events (the discrimination regime: Eq. 4's radial
     * and pulse-shape information binned against energy instead of as 1D marginals).
     * Slice b of the 2D energy x radius histogram is the energy window of the events in
     * radial bin b (rad_class and the radial geometry as for n_rad), likewise for pulse
     * shape.  Species templates s_k[i] q_k[b] (1 + field_amp u[i][b]), normalised per
     * species over each slice set; Eq. 2 on every slice.  Requires BX_FP32 or BX_BF16X3, n_rad = n_psd = 0
     * and n_rad2d + n_psd2d + 1 + (tag_frac != NULL) <= 128 slices; all toys of a model
     * are either 2D or not. */
    int n_rad2d;                /* radial slices over [0, r_fid) (0: no energy x radius histogram) */
    int n_psd2d;                /* pulse-shape slices (0: no energy x pulse-shape histogram) */
    const double* psd2d_prob;   /* [K][n_psd2d] pulse-shape bin probabilities */
    const double* field2d;      /* [N][n_rad2d + n_psd2d] template modulation u, |u| <= 1 */
    double field_amp;           /* 0 <= field_amp < 1 */
    const double* counts_rad2d; /* [n_rad2d][m_hi - m_lo] */
    const double* counts_psd2d; /* [n_psd2d][m_hi - m_lo] */
    /* Species-specific quenching (alpha or gamma species quench differently from electrons,
     * Eq. 1's Birks parameter): species k quenches with kB * quench[k] on the same
     * stopping-power table.  The species are grouped by multiplier (at most 4 groups), and
     * every group has its own Birks map and response columns.  More than one group requires
     * BX_FP32 or BX_FP64 and no 2D histograms, and needs (groups - 1) * ceil(n_grid / 128) * 128
     * + n_grid <= 8192 columns. */
    const double* quench;       /* [K] Birks multiplier per species (>= 0), or NULL: 1 for all */
    /* Energy slices of the Eq. 4 terms (its sums over several radial and pulse-shape terms):
     * slice s covers the window bins [eslice_edges[s], eslice_edges[s+1]) (window-relative,
     * eslice_edges[0] = 0, eslice_edges[n_eslice] = m_hi - m_lo, strictly rising).  Each slice
     * has its own radial and pulse-shape histogram: A_k^(s), the TFC-vetoed events of
     * species k in the slice after pile-up, times the species' bin probabilities (the same
     * in every slice).  counts_rad is then [n_eslice][n_rad] and counts_psd
     * [n_eslice][n_psd].  n_eslice = 0 (or 1 with edges {0, m_hi - m_lo}) is one slice, the
     * whole window.  At most 4 slices, n_eslice * n_rad <= 256 and n_eslice * n_psd <= 256;
     * more than one slice requires BX_FP32 or BX_FP64 and no 2D histograms. */
    int n_eslice;
    const int* eslice_edges;    /* [n_eslice + 1], or NULL with n_eslice = 0 */
    /* The 2D slices as the joint grid of radius and pulse shape (the energy x radius x
     * pulse-shape fit of the paper's multi-dimensional outlook): with joint2d = 1, slice
     * (rho, j) = rho * n_psd2d + j of the n_rad2d x n_psd2d grid is the energy window of the
     * TFC-vetoed events in radial bin rho and pulse-shape bin j.  Templates
     * s_k[i] p_k[rho] q_k[j] (1 + field_amp u[i][(rho, j)]), normalised per species over the
     * grid.  Needs n_rad2d >= 1, n_psd2d >= 1 and n_rad2d * n_psd2d + 1 + (tag_frac != NULL)
     * <= 128; field2d is [N][n_rad2d * n_psd2d], counts_rad2d [n_rad2d * n_psd2d][m_hi - m_lo]
     * and counts_psd2d is not read. */
    int joint2d;
    /* A non-Gaussian response (of the kind the paper's outlook plans for Eq. 1): the
     * Gram-Charlier series of the Gaussian with skewness
     * resp_skew and excess kurtosis resp_kurt, density
     *   phi(z) [1 + resp_skew/6 He3(z) + resp_kurt/24 He4(z)],  He3 = z^3 - 3z, He4 = z^4 - 6z^2 + 3,
     * so the mean (LY Q) and variance (a mu + b mu^2 + c) of the response stay those of Eq. 1.
     * Bin masses from its closed-form CDF Phi(z) - phi(z) [resp_skew/6 (z^2 - 1) + resp_kurt/24
     * (z^3 - 3z)], normalised to the mass above 0 npe (BX_FP32: the generator's three quadrature
     * nodes, each density times the polynomial factor; the adjoint row by row).  0, 0: the
     * Gaussian.  Otherwise BX_FP64 or BX_FP32, no 2D histograms, and the density must stay
     * non-negative within band_sigmas. */
    double resp_skew, resp_kurt;
    /* A position-dependent response (the other response variant of the paper's outlook for
     * Eq. 1; reading: the light yield depends on where an event happens).  The fiducial volume
     * is cut into n_shell radial shells; events in shell rho see the light yield LY shell_ly[rho]
     * (same a, b, c, kB), and species k puts the fixed fraction shell_frac[k][rho] of its events
     * into shell rho (e.g. uniform in volume for internal species, near the vessel for external
     * ones; the rows normally sum to 1), so its spectrum becomes
     *   v_k[m] = sum_rho shell_frac[k][rho] sum_i R_rho[m,i] s_k[i],
     * R_rho Eq. 1's response with mu_i = LY shell_ly[rho] Q_i.  Every shell has its own response
     * columns.  0 = off; 1 <= n_shell <= 4 requires BX_FP32 or BX_FP64, no 2D histograms, a single
     * Birks multiplier (quench NULL or all equal), one energy estimator, and
     * (n_shell - 1) * ceil(n_grid / 128) * 128 + n_grid <= 8192 columns. */
    int n_shell;
    const double* shell_ly;     /* [n_shell] light-yield factor of each shell (> 0) */
    const double* shell_frac;   /* [K][n_shell] fraction of species k's events in each shell (>= 0) */
} bx_model_desc;

typedef struct {
    int precision;              /* bx_precision */
    int max_batch;              /* largest n of bx_nll_batch / bx_fit (>= 1) */
    double band_sigmas;         /* response entries with |m w - mu_i| > band_sigmas sigma_i
                                   are skipped (their mass is < 1e-15); 0 -> 8 */
    double watchdog_s;          /* time budget of any device-side wait; 0 -> 2 s */
} bx_options;

/* Create a model of n_toys datasets (arrays copied to the device).  opts may be NULL
 * (BX_FP32, max_batch 1).  cuda_stream is a cudaStream_t (NULL = legacy default). */
int bx_model_create(const bx_model_desc* descs, int n_toys, const bx_options* opts,
                    void* cuda_stream, bx_model** out);
/* (bx_model_create returns BX_EINVAL, with the sizes in bx_last_error, when one item's
 * assembly stage would need more shared memory than the device allows a thread block: it
 * holds the window's spectra, the full axis of Eq. 3 spectra, the pile-up spectrum and the
 * per-column Eq. 4 weights.  On a GB300 that bounds e.g. an 8192-point grid to an axis of
 * about 2000 bins; the 1D limits above are the upper bounds of each size alone.) */
/* Several energy estimators of each dataset, fitted jointly (Sec. 3: the charge, the number of
 * detected photons and the number of fired channels are each an observable N_x with its own
 * response R_x of Eq. 1).  descs holds n_data x n_est descriptions, dataset-major: descs[t n_est + e]
 * is estimator e of dataset t, with its own bin width, window, random-trigger spectrum and data.
 * The estimators of a dataset share the events, so their grids, species shapes, stopping power,
 * tag fractions and quenching must be identical (BX_EINVAL otherwise); only estimator 0 may carry
 * the radial and pulse-shape terms, and none 2D histograms or energy slices; 1 <= n_est <= 4.
 * The rates, kB, eps and s_r are shared; each estimator has its own LY, a, b, c.  Every call then
 * takes datasets as toys (toy_idx in [0, n_data)) and the joint parameter vector
 *   theta = [r_0 .. r_{K-1}, LY_0, a_0, b_0, c_0, kB, eps, s_r, LY_1, a_1, b_1, c_1, ..., c_{n_est-1}]
 * (P = K + 7 + 4 (n_est - 1); n_est = 1 is bx_model_create): -lnL is the sum of the estimators'
 * -lnL (each evaluated at [r, LY_e, a_e, b_e, c_e, kB, eps, s_r]), its gradient is in the joint
 * layout, bx_expected returns the estimators' bins one estimator after the other, and bx_fit fits
 * the joint vector (free_mask, lo, hi in the joint layout of the largest K).  max_batch counts
 * datasets; the workspace holds max_batch x n_est evaluation items. */
int bx_model_create_estimators(const bx_model_desc* descs, int n_data, int n_est, const bx_options* opts,
                               void* cuda_stream, bx_model** out);
void bx_model_destroy(bx_model* model);
int bx_model_set_stream(bx_model* model, void* cuda_stream);
/* P = 7 + max_t K_t: the row stride of every theta / grad array */
int bx_model_n_params(const bx_model* model);
/* bins of toy t: window (+ window if tagged) + slices * (n_rad + n_psd) + B2 window, with
 * B2 = n_rad2d + n_psd2d, or n_rad2d * n_psd2d for the joint grid */
int bx_model_n_bins(const bx_model* model, int toy);
/* Sticky device status (BX_OK or BX_ETIMEOUT) after synchronising the model's stream. */
int bx_model_status(bx_model* model);

/* Stage timing.  Every call returns, for the evaluations recorded since the previous call,
 * the per-stage device times summed over them (stage_ms[5]: per-column preparation,
 * response forward, spectra/pile-up/-lnL assembly, adjoint, gather; NULL to skip), their
 * number (*n_evals) and the number of in-band response entries (pairs of output bin and
 * true-energy point within band_sigmas of the mean) they evaluated (*entries); it then
 * clears the record and switches recording on (enable = 1) or off (0).  Recording puts CUDA
 * events between the kernels on the model's stream and counts entries in the preparation
 * kernel.  Synchronises the stream. */
int bx_model_profile(bx_model* model, int enable, double* stage_ms, int* n_evals, double* entries);

/* -lnL of toy 0 at theta[P] (host arrays). */
int bx_nll(bx_model* model, const double* theta, double* nll);
/* -lnL and its gradient grad[P] of toy 0 (host arrays).  The gradient comes from the
 * hand-written adjoint (the paper minimises with numerical derivatives instead). */
int bx_nll_grad(bx_model* model, const double* theta, double* nll, double* grad);
/* Expected counts of every bin of toy `toy` at theta (host arrays), in the order:
 * vetoed window, tagged window, radial, pulse shape. */
int bx_expected(bx_model* model, int toy, const double* theta, double* mu);
/* n independent evaluations: item j uses toy toy_idx[j] (host array; NULL = toy 0 for
 * every item) at theta[j*P .. j*P + P_t).  nll[n]; grad[n*P] or NULL (no adjoint).
 * device_ptrs = 0: theta/nll/grad are host memory, synchronous.
 * device_ptrs = 1: theta/nll/grad are device memory; the call only enqueues work.
 * n = 0 is an empty batch: BX_OK, nothing is read or written. */
int bx_nll_batch(bx_model* model, int n, const int* toy_idx, const double* theta,
                 double* nll, double* grad, int device_ptrs);

/* Batched fits (the minimisation of Sec. 4; the paper uses TMinuit with numerical
 * derivatives of -lnL).  Damped Newton iterations driven by the adjoint gradient: at every
 * iterate the Hessian is re-measured by central differences of the gradient (all 2 n_free
 * displaced points in one batched evaluation) and inverted with the smallest Levenberg
 * damping that makes it positive definite; the line search evaluates 8 step lengths
 * (1 .. 1/128, within a trust region of the response, pile-up and radial parameters) in one
 * batched evaluation and takes the one with the lowest -lnL among those with sufficient
 * decrease.  Each fit in flight
 * occupies 8 + 2P evaluation slots (max_batch >= 8 + 2P).  Converged when EDM = g^T V g / 2 <
 * tol_edm with a fresh, at most lightly damped Hessian.  With BX_FP32 the gradient noise sets an
 * EDM floor and the tolerance used is max(tol_edm, 1e-5) (distance to the optimum < ~0.005
 * sigma); an FP64 model started at the FP32 optimum refines it in a few iterations.
 * The n fits run as one persistent launch: a device work queue feeds F fits in flight (F <=
 * max_batch / (8 + 2P)); when a fit finishes its result is stored and its slots take the next
 * fit of the queue, on the device.  The rounds run inside one CUDA graph whose conditional
 * loop the device ends when no fit is active or a budget is spent (the evaluation budget, or
 * time_budget_s of wall time on the device clock: unfinished fits then report BX_ETIMEOUT).  F
 * is the caller's fits_in_flight, or the autotuner's choice: it times one evaluation round for
 * F = the largest feasible value and its halves, and for each forward tile shape of the model,
 * on the fits' own datasets, and takes the largest F within 10% of the best rate; the choice is
 * kept for further calls of the same size and is reported by bx_fit_last_plan.
 * Steps: the 8 trial lengths of a line search are evaluated together and the best point with
 * sufficient decrease is taken; each non-rate component of a step is clipped to
 * max(|theta_i|, 3 sigma_i).  A BX_FP32 fit whose fresh Hessian is indefinite while no trial
 * lowers -lnL retakes the Hessian with 4x larger steps, and past 64 conditional deviations
 * stops with BX_OK at its noise floor.  A damping runaway (no damping up to 1e8 helps) retakes
 * the Hessian with 4x larger steps, at most 3 times, before the fit ends with BX_ENOTCONV; a fit
 * still running after every 25 accepted steps doubles its finite-difference step. */
typedef struct {
    double tol_edm;             /* EDM tolerance (0 -> 1e-8) */
    int max_iter;               /* evaluation budget per fit (0 -> 5000) */
    const unsigned char* free_mask; /* [P] 1 = free (NULL: all free except s_r without radial term) */
    const double* lo;           /* [P] lower bounds (NULL: rates >= 0, LY >= 50, a, b, kB >= 0,
                                   c >= 1e-3, eps in [0, 1], s_r >= 0.05) */
    const double* hi;           /* [P] upper bounds (NULL: eps <= 1, otherwise none) */
    int iters_per_launch;       /* evaluation rounds per graph replay (0 -> 4) */
    double* cov_out;            /* [n][P][P] host, or NULL: per fit the inverse Hessian of -lnL
                                   at the last fresh Hessian (the covariance of the estimates at a
                                   converged fit); rows and columns of fixed parameters and of
                                   parameters held at a bound are 0 */
    double time_budget_s;       /* device-clock budget of the whole batch (0 -> 300 s) */
    int fits_in_flight;         /* fits run concurrently by the work queue (0: autotuned) */
} bx_fit_opts;
/* free_mask/lo/hi are given in the layout of a toy with max K species: slots 0..Kmax-1 are
 * rates, Kmax..Kmax+6 the seven response/pile-up/radial parameters (then LY, a, b, c of every
 * further energy estimator of a bx_model_create_estimators model); a toy with K_t < Kmax
 * species uses its first K_t rate slots. */

typedef struct {
    double nll;                 /* -lnL at the returned theta */
    double edm;                 /* estimated distance to minimum */
    int iters;                  /* accepted Newton steps */
    int n_evals;                /* NLL+gradient evaluations used */
    int status;                 /* BX_OK, BX_ENOTCONV, BX_EDOMAIN or BX_ETIMEOUT (time budget spent) */
    int n_at_bound;             /* free parameters held at a bound at the returned theta: on the
                                   bound with the gradient pointing out of the box, so outside the
                                   Newton step (a parameter resting on a bound with an inward or
                                   zero gradient is not counted) */
    double damping;             /* Levenberg damping of the last fresh Hessian (scaled units;
                                   0: positive definite as measured) */
} bx_fit_result;

/* The launch plan of the last bx_fit call on a model. */
typedef struct {
    int fits;                   /* fits of the call */
    int fits_in_flight;         /* F: fits the work queue kept running at once (the wave shape) */
    int slots_per_fit;          /* evaluation items per fit in flight: 8 + 2P */
    int iters_per_launch;       /* evaluation rounds per pass of the graph's loop body */
    int graph_launches;         /* host launches of the batch (1) */
    int rounds;                 /* evaluation rounds the device loop ran */
    int fwd_tile;               /* forward tile shape chosen by the autotuner (0: 128-row CTAs,
                                   1: 64-row CTAs of the FP32 forward; -1: not tuned) */
    double tuned_evals_per_s;   /* evaluation throughput of the chosen shape when it was tuned */
} bx_fit_plan;
int bx_fit_last_plan(const bx_model* model, bx_fit_plan* out);

/* n fits; item j fits toy toy_idx[j] (host, NULL = toy 0) from theta0[j*P..].
 * theta_out[n*P], res[n] (host).  Returns BX_OK when every fit converged, otherwise the
 * first non-OK per-fit status (the results are filled in either case). */
int bx_fit(bx_model* model, int n, const int* toy_idx, const double* theta0,
           const bx_fit_opts* opts, double* theta_out, bx_fit_result* res);

/* Diagnostic of the tensor-core path: multiplies a 128 x 32 FP32 matrix by a 16 x 32 one
 * through the same three-part operand split (hi on a per-row power-of-two grid, TF32 mid and
 * lo), shared-memory operand layout, tcgen05.mma issue and tensor-memory drain as the forward
 * kernel, on the current device, and returns the largest relative error against an FP64 host
 * product in *max_rel_err (expected ~1e-7). */
int bx_selftest_tensor_core(double* max_rel_err);
/* Diagnostic of the device watchdog: launches one warp that waits on an mbarrier nothing
 * ever arrives on, bounded by budget_s (0 < budget_s <= 10).  Returns BX_ETIMEOUT when the
 * wait ran out as designed (the CUDA context stays usable), BX_ECUDA on a CUDA error. */
int bx_selftest_watchdog(double budget_s);

/* Allocation-free forward stage, for callers that cannot call cudaMalloc: a host process
 * whose device memory belongs to another allocator or a budget fixed at start-up, a loop
 * where cudaMalloc's implicit synchronisation would stall other streams, or a host that
 * forbids allocation after initialisation.  (The paper has no counterpart; this is a
 * deployment convenience.)
 * Computes the Eq. 3 energy spectra before pile-up of one dataset at one parameter point,
 *   lambda_h[m] = sum_i R[m,i] sum_k r_k c_{h,k} s_k[i],  m in [0, m_hi),
 * with the same FP32 kernels as BX_FP32 (vetoed spectrum in lambda[0..m_hi), tagged in
 * lambda[m_hi..2 m_hi) when tag_frac is given).  Every pointer is device memory owned by the
 * caller: shapes [K][n_grid], stop_pow [n_grid], tag_frac [K] or NULL, theta [K + 7],
 * lambda [m_hi] or [2][m_hi].  Limits of the fixed scratch: n_grid <= 4096, m_hi <= 4096,
 * K <= 16 (BX_EINVAL beyond).  The work is enqueued on cuda_stream and the call returns.
 * Its scratch is one 530 KiB static device array per device, whose address is looked up on
 * the first call made on that device; all calls share
 * it, so calls that overlap on the GPU race.  A parameter point outside the model's domain
 * (non-finite theta, LY <= 0, sigma^2 <= 0 at a grid point) fills lambda with NaN; the call
 * itself still returns BX_OK, because the check runs on the device after it has returned. */
int bx_spectra_noalloc(int n_grid, double e_max, int n_species, const double* shapes,
                       const double* stop_pow, const double* tag_frac, double width, int m_hi,
                       const double* theta, double* lambda, void* cuda_stream);

/* Ceilings of the roofline (measurement tools; the paper has no counterpart).  Runs one
 * input-free microkernel on the current device, on cuda_stream, over a grid of whole waves
 * (every SM full), after one shorter warm-up launch, and returns its CUDA-event time in *ms
 * and the units it completed in *units:
 *   BX_CEIL_RESP      response entries of the FP32 bin-mass routine of the forward (Eq. 1,
 *                     3-point Gauss-Legendre, the branch of in-band entries) alone;
 *   BX_CEIL_RESP_ACC  response entries with the forward's accumulation per entry (two
 *                     compensated row sums and one column-sum FMA);
 *   BX_CEIL_FMA64     FP64 floating-point operations (FMA = 2);
 *   BX_CEIL_FMA32     FP32 floating-point operations (FMA = 2).
 * reps (1 .. 2^20) scales the work: 512 entries, or 1024 flops, per thread and rep.
 * Allocates and frees a small device buffer; synchronises the stream. */
enum { BX_CEIL_RESP = 0, BX_CEIL_RESP_ACC = 1, BX_CEIL_FMA64 = 2, BX_CEIL_FMA32 = 3 };
int bx_ceiling(int which, int reps, void* cuda_stream, double* ms, double* units);

const char* bx_last_error(void);
const char* bx_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* BX_H */
