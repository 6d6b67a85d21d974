/*
 * bx_oracle.c -- plain, slow, FP64 CPU oracle of the binned Poisson -lnL of the
 * Borexino-style multivariate spectral fit (arXiv:1805.11125, Sec. 3, Eq. 1-4).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Every quantity is computed literally from its definition, dense over every
 * (output bin m, true-energy point i) pair (no band cut), in double precision:
 *
 *   a1  Birks/light-yield map (Eq. 1 "parameters p0, p1, ..."; the paper gives no form,
 *       reading: Birks quenching on a caller-supplied stopping-power table)
 *         Q_i   = sum_{j<i} dE/(1 + kB S_j) + dE/(2 (1 + kB S_i))
 *         mu_i  = LY Q_i,      sigma_i^2 = a mu_i + b mu_i^2 + c
 *       with species-specific quenching (the "next" response variant: alpha or gamma
 *       species quench differently) species k uses kB quench[k]; the species are grouped by
 *       multiplier and every group has its own map and response (a2)
 *       with a position-dependent response (the "next" response variant; reading: the light
 *       yield depends on where in the detector an event happens, the fiducial volume is cut
 *       into radial shells, shell rho has the light yield LY f_rho, and species k puts the
 *       fixed fraction q_k[rho] of its events into shell rho) every shell has its own map and
 *       response, and v_k[m] = sum_rho q_k[rho] sum_i R_rho[m,i] s_k[i] in a3
 *   a2  response of Eq. 1, bin-integrated Gaussian in npe, normalised to the mass above 0:
 *         R[m,i] = (Phi(z_{m+1,i}) - Phi(z_{m,i})) / Phi(mu_i / sigma_i),
 *         z_{m,i} = (m w - mu_i) / sigma_i
 *   a3  v_k[m] = sum_i R[m,i] s_k[i]                                   (Eq. 1)
 *   a4  lambda_h[m] = sum_k r_k c_{h,k} v_k[m]; TFC-vetoed c = 1 - t_k, tagged c = t_k
 *       (Eq. 3); radial / pulse-shape terms are window marginals A_k of the TFC-vetoed
 *       species spectra times bin probabilities (Eq. 4)
 *   a5  pile-up (Eq. 2 with the scale eps):
 *         mu_h[m] = (1 - eps) lambda_h[m] + eps sum_{d=0}^{min(m, L-1)} g[d] lambda_h[m-d]
 *   a6  -lnL = sum over all bins of  mu - n + n ln(n / mu)   (n ln(n/mu) := 0 at n = 0),
 *       summed with Neumaier compensation                     (Eq. 3, Eq. 4)
 *   2D  (the discrimination regime: Eq. 4's radial and pulse-shape information as 2D
 *       energy x radius and energy x pulse-shape histograms instead of 1D marginals;
 *       reading: templates s_k[i] q_k[b] (1 + amp u[i,b]) with the caller's smooth field u,
 *       normalised per species over each slice set)
 *         T_r[i,b] = sum_k r_k (1 - t_k) s_k[i] q_k[b] (1 + amp u[i,b]) / N_k(set of b)
 *         Y[m,b]   = sum_i R[m,i] T_r[i,b],  then Eq. 2 on every slice b
 *       with q_k[b] the radial bin probability of slice b (internal / external as for the
 *       radial term) or the pulse-shape bin probability.
 *   3D  (the joint energy x radius x pulse-shape fit, the paper's multi-dimensional outlook):
 *       the same with one slice per cell (rho, j) of the radius x pulse-shape grid,
 *       q_k[(rho, j)] = p_k[rho] ps_k[j], normalised per species over the whole grid.
 *
 * Gradients come from forward-mode dual numbers carried through the same definition
 * (independent of any hand-written adjoint).  The fit is a damped Newton iteration on
 * the dual-number gradient with a central-difference Hessian, box bounds by projection.
 * The fit is pinned by two invariants (an Asimov fit returns theta_true; at the optimum
 * the expected and observed totals agree) and one closed form (a single free rate of a
 * one-species model ends at sum(n) / sum(u) on any data); beyond them its parity is
 * unpinned: the paper prints no fitted values.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OPMAX 40                       /* max parameters (K <= 33) */

typedef struct { double v; double d[OPMAX]; } dual;

static int NP = 0;                     /* active derivative slots for the current call */

static inline dual dc(double x) { dual r; r.v = x; memset(r.d, 0, sizeof r.d); return r; }
static inline dual dvar(double x, int j) { dual r = dc(x); if (j >= 0 && j < NP) r.d[j] = 1.0; return r; }
static inline dual dadd(dual a, dual b) { dual r; r.v = a.v + b.v; for (int j = 0; j < NP; ++j) r.d[j] = a.d[j] + b.d[j]; return r; }
static inline dual dsub(dual a, dual b) { dual r; r.v = a.v - b.v; for (int j = 0; j < NP; ++j) r.d[j] = a.d[j] - b.d[j]; return r; }
static inline dual dmul(dual a, dual b) { dual r; r.v = a.v * b.v; for (int j = 0; j < NP; ++j) r.d[j] = a.d[j] * b.v + a.v * b.d[j]; return r; }
static inline dual dscale(dual a, double s) { dual r; r.v = a.v * s; for (int j = 0; j < NP; ++j) r.d[j] = a.d[j] * s; return r; }
static inline dual dshift(dual a, double s) { a.v += s; return a; }
static inline dual ddiv(dual a, dual b) {
    dual r; r.v = a.v / b.v;
    for (int j = 0; j < NP; ++j) r.d[j] = (a.d[j] - r.v * b.d[j]) / b.v;
    return r;
}
/* r = f(a) with f'(a) = fp */
static inline dual dfun(dual a, double f, double fp) { dual r; r.v = f; for (int j = 0; j < NP; ++j) r.d[j] = fp * a.d[j]; return r; }
static inline dual dexp(dual a) { double e = exp(a.v); return dfun(a, e, e); }
static inline dual dlog(dual a) { return dfun(a, log(a.v), 1.0 / a.v); }
static inline dual dsqrt(dual a) { double s = sqrt(a.v); return dfun(a, s, 0.5 / s); }
static const double SQRT1_2 = 0.70710678118654752440;
static const double INV_SQRT_2PI = 0.39894228040143267794;
/* standard normal lower tail Phi(x) and upper tail Q(x) = 1 - Phi(x), both via erfc */
static inline dual dPhi(dual x) { return dfun(x, 0.5 * erfc(-x.v * SQRT1_2), INV_SQRT_2PI * exp(-0.5 * x.v * x.v)); }
static inline dual dQ(dual x) { return dfun(x, 0.5 * erfc(x.v * SQRT1_2), -INV_SQRT_2PI * exp(-0.5 * x.v * x.v)); }
/* accumulate a += s * b */
static inline void daxpy(dual* a, double s, const dual* b) { a->v += s * b->v; for (int j = 0; j < NP; ++j) a->d[j] += s * b->d[j]; }
static inline void dacc(dual* a, dual b) { a->v += b.v; for (int j = 0; j < NP; ++j) a->d[j] += b.d[j]; }

/* Gaussian mass in [za, zb] (za < zb), evaluated on the tail away from the mean so that
 * no significant digits cancel: the plain definition Phi(zb) - Phi(za). */
static dual gauss_mass(dual za, dual zb) {
    if (za.v >= 0.0) return dsub(dQ(za), dQ(zb));
    if (zb.v <= 0.0) return dsub(dPhi(zb), dPhi(za));
    return dsub(dsub(dc(1.0), dQ(zb)), dPhi(za));
}


typedef struct {
    int n_grid; double e_max;
    int K; const double* shapes;       /* [K][n_grid] */
    const double* stop_pow;            /* [n_grid] MeV/cm */
    const double* tag_frac;            /* [K] or NULL (single spectrum) */
    int L; const double* pileup;       /* [L] */
    double width; int m_lo, m_hi;      /* window [m_lo, m_hi) on the axis [0, m_hi) */
    const double* n_sub;               /* [m_hi - m_lo] */
    const double* n_tag;               /* [m_hi - m_lo] or NULL */
    int n_rad; const int* rad_class;   /* [K]: 0 internal, 1 external; n_rad = 0 -> none */
    double r_fid, r_iv, att_len;
    const double* n_rad_counts;        /* [n_rad] */
    int n_psd; const double* psd_prob; /* [K][n_psd]; n_psd = 0 -> none */
    const double* n_psd_counts;        /* [n_psd] */
    int n_r2, n_p2;                    /* 2D slices: radial (uses rad_class), pulse shape */
    const double* field;               /* [n_grid][n_r2 + n_p2] */
    double amp;
    const double* psd2;                /* [K][n_p2] */
    const double* n_r2_counts;         /* [n_r2][m_hi - m_lo] */
    const double* n_p2_counts;         /* [n_p2][m_hi - m_lo] */
    const double* quench;              /* [K] Birks multiplier per species (species k quenches with
                                          kB quench[k]); NULL -> 1 for every species */
    int n_es; const int* es_edges;     /* energy slices of Eq. 4 (its sums over radial and
                                          pulse-shape terms): slice s is the window bins
                                          [es_edges[s], es_edges[s+1]), edges from 0 to m_hi - m_lo;
                                          n_es = 0 -> one slice, the whole window.  The radial and
                                          pulse-shape counts are then [n_es][n_rad], [n_es][n_psd] */
    double gc_skew, gc_kurt;           /* Gram-Charlier response (a non-Gaussian response of the kind
                                          the paper's outlook plans): skewness gamma_1 and excess
                                          kurtosis gamma_2 of the photoelectron response; 0, 0 is the
                                          Gaussian */
    int joint2;                        /* 2D slices as the joint grid of radius and pulse shape:
                                          slice (rho, j) = rho n_p2 + j of the n_r2 x n_p2 grid is the
                                          energy window of the events in radial bin rho and pulse-shape
                                          bin j (the energy x radius x pulse-shape histogram); field
                                          [n_grid][n_r2 n_p2], counts in n_r2_counts [n_r2 n_p2][nw] */
    int n_shell;                       /* position-dependent response: radial shells (0: none) */
    const double* shell_ly;            /* [n_shell] light-yield factor f_rho of each shell (> 0) */
    const double* shell_frac;          /* [K][n_shell] fraction q_k[rho] of species k's events in
                                          shell rho (>= 0) */
} om_model;

/* Gram-Charlier (type A) response (reading: the non-Gaussian response of the paper's outlook,
 * with the paper's mean and variance kept):
 *   f(z) = phi(z) [1 + g1/6 He3(z) + g2/24 He4(z)],  He3 = z^3 - 3z, He4 = z^4 - 6z^2 + 3,
 * whose mean, variance, skewness and excess kurtosis are 0, 1, g1, g2 (He3, He4 are orthogonal
 * to 1, z, z^2 under phi).  Since d/dz [phi He_{n-1}] = -phi He_n, its CDF is
 *   F(z) = Phi(z) - phi(z) [g1/6 He2(z) + g2/24 He3(z)],  He2 = z^2 - 1,
 * so a bin's mass is the Gaussian mass minus the difference of phi(z) C(z),
 * C(z) = g1/6 He2(z) + g2/24 He3(z), at its edges. */
static dual gc_term(const om_model* m, dual z) {   /* phi(z) C(z) */
    dual z2 = dmul(z, z);
    dual he2 = dshift(z2, -1.0), he3 = dsub(dmul(z2, z), dscale(z, 3.0));
    dual Cz = dadd(dscale(he2, m->gc_skew / 6.0), dscale(he3, m->gc_kurt / 24.0));
    dual phi = dscale(dexp(dscale(z2, -0.5)), INV_SQRT_2PI);
    return dmul(phi, Cz);
}
static int gc_on(const om_model* m) { return m->gc_skew != 0.0 || m->gc_kurt != 0.0; }
static dual resp_mass(const om_model* m, dual za, dual zb) {
    dual g = gauss_mass(za, zb);
    return gc_on(m) ? dsub(g, dsub(gc_term(m, zb), gc_term(m, za))) : g;
}
/* mass above 0 npe of the response of mean mu and width sig: 1 - F(-mu/sig) */
static dual resp_above0(const om_model* m, dual mu, dual sig) {
    dual x = ddiv(mu, sig);
    dual base = dPhi(x);
    return gc_on(m) ? dadd(base, gc_term(m, dscale(x, -1.0))) : base;
}

enum { OM_MAX_SETS = 4 };

/* Species-specific quenching (reading: a species' Birks constant is kB times its own
 * multiplier, e.g. ~1e2 for alpha particles on the electron stopping-power table): the species
 * are grouped by multiplier, and each group ("set") has its own Birks map and response.
 * Returns the number of sets (<= OM_MAX_SETS, 0 if there are more), their multipliers xi[]
 * and each species' set in set_of[]. */
static int quench_sets(const om_model* m, double* xi, int* set_of) {
    int n = 0;
    for (int k = 0; k < m->K; ++k) {
        const double q = m->quench ? m->quench[k] : 1.0;
        int c = 0;
        while (c < n && xi[c] != q) ++c;
        if (c == n) {
            if (n == OM_MAX_SETS) return 0;
            xi[n++] = q;
        }
        set_of[k] = c;
    }
    return n;
}

enum { OM_OK = 0, OM_EINVAL = -1, OM_ENOMEM = -2, OM_EDOMAIN = -4, OM_ENOTCONV = -6 };

int om_n_params(const om_model* m) { return m->K + 7; }

static int n_slices(const om_model* m) { return m->n_es > 0 ? m->n_es : 1; }

/* number of 2D slices: the radial and pulse-shape sets, or their joint grid */
static int n_slices2(const om_model* m) { return m->joint2 ? m->n_r2 * m->n_p2 : m->n_r2 + m->n_p2; }

int om_n_bins(const om_model* m) {
    int nw = m->m_hi - m->m_lo, S = n_slices(m);
    return nw + (m->tag_frac ? nw : 0) + S * (m->n_rad > 0 && m->rad_class ? m->n_rad : 0) +
           S * (m->n_psd > 0 && m->psd_prob ? m->n_psd : 0) + n_slices2(m) * nw;
}

static int check_model(const om_model* m) {
    if (!m || m->n_grid < 1 || m->K < 1 || m->K + 7 > OPMAX || m->L < 1 || m->width <= 0 ||
        m->m_lo < 0 || m->m_hi <= m->m_lo || !m->shapes || !m->stop_pow || !m->pileup)
        return OM_EINVAL;
    if (m->n_r2 < 0 || m->n_p2 < 0 || (m->n_r2 + m->n_p2 > 0 && !m->field) || (m->n_r2 > 0 && !m->rad_class) ||
        (m->n_p2 > 0 && !m->psd2))
        return OM_EINVAL;
    if (m->joint2 && (m->n_r2 < 1 || m->n_p2 < 1)) return OM_EINVAL;   /* the joint grid needs both axes */
    if (m->quench) {
        for (int k = 0; k < m->K; ++k)
            if (!(m->quench[k] >= 0.0) || !isfinite(m->quench[k])) return OM_EINVAL;
        double xi[OM_MAX_SETS];
        int set_of[OPMAX];
        const int n = quench_sets(m, xi, set_of);
        if (n == 0 || (n > 1 && m->n_r2 + m->n_p2 > 0)) return OM_EINVAL;   /* 2D slices: one set only */
    }
    if (m->n_es < 0 || (m->n_es > 0 && (!m->es_edges || m->n_r2 + m->n_p2 > 0))) return OM_EINVAL;
    if (m->n_shell < 0 || m->n_shell > OM_MAX_SETS) return OM_EINVAL;
    if (m->n_shell > 0) {   /* shells: 1D histograms and one Birks multiplier only */
        if (!m->shell_ly || !m->shell_frac || m->n_r2 + m->n_p2 > 0) return OM_EINVAL;
        double xi[OM_MAX_SETS];
        int set_of[OPMAX];
        if (quench_sets(m, xi, set_of) != 1) return OM_EINVAL;
        for (int r = 0; r < m->n_shell; ++r)
            if (!(m->shell_ly[r] > 0.0) || !isfinite(m->shell_ly[r])) return OM_EINVAL;
        for (int j = 0; j < m->K * m->n_shell; ++j)
            if (!(m->shell_frac[j] >= 0.0) || !isfinite(m->shell_frac[j])) return OM_EINVAL;
    }
    if (m->n_es > 0) {   /* the slices partition the window */
        if (m->es_edges[0] != 0 || m->es_edges[m->n_es] != m->m_hi - m->m_lo) return OM_EINVAL;
        for (int q = 0; q < m->n_es; ++q)
            if (m->es_edges[q + 1] <= m->es_edges[q]) return OM_EINVAL;
    }
    return OM_OK;
}

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) { double p3 = p2; p2 = p1; p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j; }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z; z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-16) break;
        }
        x[i] = -z; x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* Radial bin probabilities (Eq. 4 radial term, reading: internal species uniform in
 * volume, external density exp(-(R_iv - r) / (att_len * s_r)) in a fiducial sphere of
 * radius r_fid): p[rho] = int_{bin} r^2 f(r) dr / int_0^{r_fid} r^2 f(r) dr, integrals by
 * 24-point Gauss-Legendre per bin. */
static void radial_probs_n(const om_model* m, int nbins, dual s_r, int cls, dual* p) {
    enum { NGL = 24 };
    double gx[NGL], gw[NGL];
    gauss_legendre(NGL, gx, gw);
    dual lam = dscale(s_r, m->att_len);
    dual tot = dc(0.0);
    double h = m->r_fid / nbins;
    for (int b = 0; b < nbins; ++b) {
        dual acc = dc(0.0);
        double c0 = (b + 0.5) * h;
        for (int q = 0; q < NGL; ++q) {
            double r = c0 + 0.5 * h * gx[q];
            double wq = 0.5 * h * gw[q] * r * r;
            dual f = cls == 1 ? dexp(ddiv(dc(-(m->r_iv - r)), lam)) : dc(1.0);
            daxpy(&acc, wq, &f);
        }
        p[b] = acc;
        tot = dadd(tot, acc);
    }
    for (int b = 0; b < nbins; ++b) p[b] = ddiv(p[b], tot);
}
static void radial_probs(const om_model* m, dual s_r, int cls, dual* p) { radial_probs_n(m, m->n_rad, s_r, cls, p); }

/* Neumaier-compensated accumulator on every dual component */
typedef struct { dual s, c; } nsum;
static void nsum_add(nsum* a, const dual* x) {
    double t = a->s.v + x->v;
    a->c.v += fabs(a->s.v) >= fabs(x->v) ? (a->s.v - t) + x->v : (x->v - t) + a->s.v;
    a->s.v = t;
    for (int j = 0; j < NP; ++j) {
        double tj = a->s.d[j] + x->d[j];
        a->c.d[j] += fabs(a->s.d[j]) >= fabs(x->d[j]) ? (a->s.d[j] - tj) + x->d[j] : (x->d[j] - tj) + a->s.d[j];
        a->s.d[j] = tj;
    }
}

/* a6 term of one bin: mu - n + n ln(n/mu) */
static int bin_term(double n, dual mu, dual* out) {
    if (n == 0.0) { *out = mu; return OM_OK; }
    if (!(mu.v > 0.0)) { *out = dc(INFINITY); return OM_EDOMAIN; }
    /* value: mu - n + n ln(n/mu), with ln(n/mu) = log1p((n - mu)/mu) so that the
     * logarithm keeps its relative precision when n is close to mu;
     * derivative: (1 - n/mu) dmu */
    dual r = dfun(mu, (mu.v - n) + n * log1p((n - mu.v) / mu.v), 1.0 - n / mu.v);
    *out = r;
    return OM_OK;
}

typedef struct {
    dual *Q, *mu, *sig, *den;          /* [N] */
    dual *v;                           /* [M][K] */
} work;

static void work_free(work* w) { free(w->Q); free(w->mu); free(w->sig); free(w->den); free(w->v); }

/* a1: quenching + light yield + resolution for the species of Birks multiplier xi (kB xi),
 * light yield LY f (f: the factor of a radial shell, else 1); returns OM_EDOMAIN if
 * sigma^2 <= 0 anywhere. */
static int stage_a1(const om_model* m, const dual* th, work* w, double xi, double f) {
    int N = m->n_grid, K = m->K;
    dual LY = dscale(th[K], f), a = th[K + 1], b = th[K + 2], c = th[K + 3], kB = dscale(th[K + 4], xi);
    double dE = m->e_max / N;
    dual run = dc(0.0);
    int st = OM_OK;
    for (int i = 0; i < N; ++i) {
        dual x = ddiv(dc(dE), dshift(dscale(kB, m->stop_pow[i]), 1.0));
        w->Q[i] = dadd(run, dscale(x, 0.5));
        run = dadd(run, x);
        w->mu[i] = dmul(LY, w->Q[i]);
        dual var = dadd(dadd(dmul(a, w->mu[i]), dmul(b, dmul(w->mu[i], w->mu[i]))), c);
        if (!(var.v > 0.0)) { st = OM_EDOMAIN; var = dc(1.0); }
        w->sig[i] = dsqrt(var);
        w->den[i] = resp_above0(m, w->mu[i], w->sig[i]);
    }
    return st;
}

/* a2 + a3: v_k[m] = sum_i R[m,i] s_k[i] for every m in [0, m_hi) and the species of set c
 * (set_of NULL: every species); with 2D slices also Y[m][b] = sum_i R[m,i] T_r[i][b]
 * (T_r: [N][B2], Y: [M][B2]).  Radial shell rho >= 0 (R the shell's response): every species
 * k gets q_k[rho] sum_i R[m,i] s_k[i] added to v_k[m] (zeroed at rho = 0). */
static void stage_a23(const om_model* m, work* w, double* R_out, const dual* Tr, dual* Y, const int* set_of, int c,
                      int rho) {
    int N = m->n_grid, K = m->K, M = m->m_hi, B2 = n_slices2(m);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < M; ++r) {
        dual* vr = w->v + (size_t)r * K;
        for (int k = 0; k < K; ++k)
            if (rho < 0 ? (!set_of || set_of[k] == c) : rho == 0) vr[k] = dc(0.0);
        if (Y) for (int b = 0; b < B2; ++b) Y[(size_t)r * B2 + b] = dc(0.0);
        for (int i = 0; i < N; ++i) {
            dual za = ddiv(dsub(dc(r * m->width), w->mu[i]), w->sig[i]);
            dual zb = ddiv(dsub(dc((r + 1) * m->width), w->mu[i]), w->sig[i]);
            dual R = ddiv(resp_mass(m, za, zb), w->den[i]);
            if (R_out) R_out[(size_t)r * N + i] = R.v;
            for (int k = 0; k < K; ++k) {
                if (rho < 0 && set_of && set_of[k] != c) continue;
                double s = m->shapes[(size_t)k * N + i];
                if (rho >= 0) s *= m->shell_frac[(size_t)k * m->n_shell + rho];
                if (s != 0.0) daxpy(&vr[k], s, &R);
            }
            if (Y)
                for (int b = 0; b < B2; ++b) dacc(&Y[(size_t)r * B2 + b], dmul(R, Tr[(size_t)i * B2 + b]));
        }
    }
}

/* Templates of the joint energy x radius x pulse-shape grid: slice b = rho n_p2 + j,
 *   T_r[i][b] = sum_k r_k (1 - t_k) s_k[i] p_k[rho] ps_k[j] (1 + amp u[i][b]) / N_k,
 *   N_k = sum_i sum_b s_k[i] p_k[rho] ps_k[j] (1 + amp u[i][b]). */
static int stage_joint_templates(const om_model* m, const dual* th, dual* Tr) {
    int N = m->n_grid, K = m->K, nR = m->n_r2, nP = m->n_p2, B2 = nR * nP;
    dual* p = calloc((size_t)nR, sizeof(dual));
    dual* q = calloc((size_t)B2, sizeof(dual));
    if (!p || !q) { free(p); free(q); return OM_ENOMEM; }
    for (size_t j = 0; j < (size_t)N * B2; ++j) Tr[j] = dc(0.0);
    for (int k = 0; k < K; ++k) {
        radial_probs_n(m, nR, th[K + 6], m->rad_class[k], p);
        for (int r = 0; r < nR; ++r)
            for (int j = 0; j < nP; ++j) q[r * nP + j] = dscale(p[r], m->psd2[(size_t)k * nP + j]);
        dual Nk = dc(0.0);
        for (int i = 0; i < N; ++i) {
            double s = m->shapes[(size_t)k * N + i];
            if (s == 0.0) continue;
            for (int b = 0; b < B2; ++b) dacc(&Nk, dscale(q[b], s * (1.0 + m->amp * m->field[(size_t)i * B2 + b])));
        }
        double ck = m->tag_frac ? 1.0 - m->tag_frac[k] : 1.0;
        dual f = ddiv(dscale(th[k], ck), Nk);
        for (int b = 0; b < B2; ++b) {
            dual coef = dmul(f, q[b]);
            for (int i = 0; i < N; ++i) {
                double x = m->shapes[(size_t)k * N + i] * (1.0 + m->amp * m->field[(size_t)i * B2 + b]);
                if (x != 0.0) daxpy(&Tr[(size_t)i * B2 + b], x, &coef);
            }
        }
    }
    free(p);
    free(q);
    return OM_OK;
}

/* 2D templates, rate-weighted: T_r[i][b] = sum_k r_k (1 - t_k) s_k[i] q_k[b] (1 + amp u[i][b]) / N_k,
 * N_k = sum_i sum_{b in the set of b} s_k[i] q_k[b] (1 + amp u[i][b]) (radial set, pulse-shape set).
 * Joint grid: q_k[(rho, j)] = p_k[rho] ps_k[j] (radial times pulse-shape probability), one set. */
static int stage_2d_templates(const om_model* m, const dual* th, dual* Tr) {
    if (m->joint2) return stage_joint_templates(m, th, Tr);
    int N = m->n_grid, K = m->K, nR = m->n_r2, nP = m->n_p2, B2 = nR + nP;
    dual* q = calloc((size_t)B2, sizeof(dual));
    if (!q) return OM_ENOMEM;
    for (size_t j = 0; j < (size_t)N * B2; ++j) Tr[j] = dc(0.0);
    for (int k = 0; k < K; ++k) {
        if (nR > 0) radial_probs_n(m, nR, th[K + 6], m->rad_class[k], q);
        for (int j = 0; j < nP; ++j) q[nR + j] = dc(m->psd2[(size_t)k * nP + j]);
        dual NR = dc(0.0), NPs = dc(0.0);
        for (int i = 0; i < N; ++i) {
            double s = m->shapes[(size_t)k * N + i];
            for (int b = 0; b < B2; ++b) {
                dual t = dscale(q[b], s * (1.0 + m->amp * m->field[(size_t)i * B2 + b]));
                if (b < nR) dacc(&NR, t); else dacc(&NPs, t);
            }
        }
        double ck = m->tag_frac ? 1.0 - m->tag_frac[k] : 1.0;
        dual fR = nR > 0 ? ddiv(dscale(th[k], ck), NR) : dc(0.0);
        dual fP = nP > 0 ? ddiv(dscale(th[k], ck), NPs) : dc(0.0);
        for (int b = 0; b < B2; ++b) {
            dual coef = dmul(b < nR ? fR : fP, q[b]);
            for (int i = 0; i < N; ++i) {
                double x = m->shapes[(size_t)k * N + i] * (1.0 + m->amp * m->field[(size_t)i * B2 + b]);
                if (x != 0.0) daxpy(&Tr[(size_t)i * B2 + b], x, &coef);
            }
        }
    }
    free(q);
    return OM_OK;
}

/* a5 on one spectrum x[0..M): y[j] = (1-eps) x[m] + eps sum_{d=0}^{min(m,L-1)} g[d] x[m-d], m = m_lo + j */
static void pileup_window(const om_model* m, dual eps, const dual* x, int stride, dual* y) {
    dual one_m_eps = dsub(dc(1.0), eps);
    for (int r = m->m_lo; r < m->m_hi; ++r) {
        dual conv = dc(0.0);
        int dmax = r < m->L - 1 ? r : m->L - 1;
        for (int d = 0; d <= dmax; ++d) daxpy(&conv, m->pileup[d], &x[(size_t)(r - d) * stride]);
        y[r - m->m_lo] = dadd(dmul(one_m_eps, x[(size_t)r * stride]), dmul(eps, conv));
    }
}

/* Full evaluation.  mu_out (values, all bins concatenated) and/or nll (+grad). */
static int evaluate(const om_model* m, const double* theta, int want_grad,
                    double* mu_out, double* nll_out, double* grad_out) {
    int st = check_model(m);
    if (st) return st;
    int N = m->n_grid, K = m->K, M = m->m_hi, P = K + 7, nw = m->m_hi - m->m_lo;
    NP = want_grad ? P : 0;
    dual th[OPMAX];
    for (int j = 0; j < P; ++j) th[j] = dvar(theta[j], j);
    dual eps = th[K + 5], s_r = th[K + 6];
    work w;
    w.Q = calloc(N, sizeof(dual)); w.mu = calloc(N, sizeof(dual)); w.sig = calloc(N, sizeof(dual));
    w.den = calloc(N, sizeof(dual)); w.v = calloc((size_t)M * K, sizeof(dual));
    int nb = om_n_bins(m);
    dual* mu = calloc(nb, sizeof(dual));
    dual* lam = calloc(M, sizeof(dual));
    dual* A = calloc((size_t)K * n_slices(m), sizeof(dual));
    dual* tmp = calloc(nw, sizeof(dual));
    const int B2 = n_slices2(m);
    dual* Tr = B2 > 0 ? calloc((size_t)N * B2, sizeof(dual)) : NULL;
    dual* Y = B2 > 0 ? calloc((size_t)M * B2, sizeof(dual)) : NULL;
    if (!w.Q || !w.mu || !w.sig || !w.den || !w.v || !mu || !lam || !A || !tmp || (B2 > 0 && (!Tr || !Y))) {
        st = OM_ENOMEM;
        goto done;
    }

    {
        double xi[OM_MAX_SETS];
        int set_of[OPMAX];
        const int nset = quench_sets(m, xi, set_of);
        if (B2 > 0 && (st = stage_2d_templates(m, th, Tr))) goto done;
        if (m->n_shell > 0) {
            for (int r = 0; r < m->n_shell; ++r) {   /* one light-yield map and response per shell */
                st = stage_a1(m, th, &w, 1.0, m->shell_ly[r]);
                if (st) goto done;
                stage_a23(m, &w, NULL, NULL, NULL, NULL, 0, r);
            }
        } else {
            for (int c = 0; c < nset; ++c) {   /* one Birks map and response per set of species */
                st = stage_a1(m, th, &w, xi[c], 1.0);
                if (st) goto done;
                stage_a23(m, &w, NULL, Tr, Y, set_of, c, -1);
            }
        }
    }

    /* a4 + a5 for the energy spectra */
    int o = 0;
    for (int h = 0; h < (m->tag_frac ? 2 : 1); ++h) {
        for (int r = 0; r < M; ++r) {
            dual s = dc(0.0);
            for (int k = 0; k < K; ++k) {
                double ck = m->tag_frac ? (h == 0 ? 1.0 - m->tag_frac[k] : m->tag_frac[k]) : 1.0;
                s = dadd(s, dscale(dmul(th[k], w.v[(size_t)r * K + k]), ck));
            }
            lam[r] = s;
        }
        pileup_window(m, eps, lam, 1, mu + o);
        o += nw;
    }
    /* Eq. 4 terms, per energy slice s: the marginal A_k^(s) of each TFC-vetoed species
     * spectrum after pile-up over the slice's window bins, times the species' radial and
     * pulse-shape bin probabilities (the same in every slice).  Radial histograms of all
     * slices first (slice-major), then the pulse-shape histograms. */
    int has_rad = m->n_rad > 0 && m->rad_class, has_psd = m->n_psd > 0 && m->psd_prob;
    const int S = n_slices(m);
    if (has_rad || has_psd) {
        for (int k = 0; k < K; ++k) {
            pileup_window(m, eps, w.v + k, K, tmp);
            double ck = m->tag_frac ? 1.0 - m->tag_frac[k] : 1.0;
            for (int q = 0; q < S; ++q) {
                const int j0 = m->n_es > 0 ? m->es_edges[q] : 0, j1 = m->n_es > 0 ? m->es_edges[q + 1] : nw;
                dual s = dc(0.0);
                for (int j = j0; j < j1; ++j) s = dadd(s, tmp[j]);
                A[(size_t)q * K + k] = dscale(dmul(th[k], s), ck);   /* vetoed events of k in slice q */
            }
        }
    }
    if (has_rad) {
        dual* p = calloc(m->n_rad, sizeof(dual));
        for (int b = 0; b < S * m->n_rad; ++b) mu[o + b] = dc(0.0);
        for (int k = 0; k < K; ++k) {
            radial_probs(m, s_r, m->rad_class[k], p);
            for (int q = 0; q < S; ++q)
                for (int b = 0; b < m->n_rad; ++b)
                    mu[o + q * m->n_rad + b] = dadd(mu[o + q * m->n_rad + b], dmul(A[(size_t)q * K + k], p[b]));
        }
        free(p);
        o += S * m->n_rad;
    }
    if (has_psd) {
        for (int q = 0; q < S; ++q)
            for (int b = 0; b < m->n_psd; ++b) {
                dual s = dc(0.0);
                for (int k = 0; k < K; ++k) s = dadd(s, dscale(A[(size_t)q * K + k], m->psd_prob[(size_t)k * m->n_psd + b]));
                mu[o + q * m->n_psd + b] = s;
            }
        o += S * m->n_psd;
    }
    /* 2D slices: Eq. 2 on every slice of Y, slice-major */
    for (int b = 0; b < B2; ++b) {
        pileup_window(m, eps, Y + b, B2, mu + o);
        o += nw;
    }
    if (mu_out) for (int j = 0; j < nb; ++j) mu_out[j] = mu[j].v;

    /* a6 */
    if (nll_out) {
        const double* cnt[6]; int len[6]; int nh = 0;
        cnt[nh] = m->n_sub; len[nh++] = nw;
        if (m->tag_frac) { cnt[nh] = m->n_tag; len[nh++] = nw; }
        if (has_rad) { cnt[nh] = m->n_rad_counts; len[nh++] = S * m->n_rad; }
        if (has_psd) { cnt[nh] = m->n_psd_counts; len[nh++] = S * m->n_psd; }
        if (m->joint2) { cnt[nh] = m->n_r2_counts; len[nh++] = B2 * nw; }
        else {
            if (m->n_r2 > 0) { cnt[nh] = m->n_r2_counts; len[nh++] = m->n_r2 * nw; }
            if (m->n_p2 > 0) { cnt[nh] = m->n_p2_counts; len[nh++] = m->n_p2 * nw; }
        }
        nsum acc; acc.s = dc(0.0); acc.c = dc(0.0);
        int jj = 0, dom = 0;
        for (int h = 0; h < nh; ++h)
            for (int j = 0; j < len[h]; ++j, ++jj) {
                if (!cnt[h]) { st = OM_EINVAL; goto done; }
                dual t;
                if (bin_term(cnt[h][j], mu[jj], &t)) dom = 1;
                else nsum_add(&acc, &t);
            }
        if (dom) { *nll_out = INFINITY; st = OM_EDOMAIN; }
        else {
            *nll_out = acc.s.v + acc.c.v;
            if (grad_out) for (int j = 0; j < P; ++j) grad_out[j] = acc.s.d[j] + acc.c.d[j];
        }
    }
done:
    work_free(&w); free(mu); free(lam); free(A); free(tmp); free(Tr); free(Y);
    return st;
}

/* ---------------------------------------------------------------- public entry points */

int om_expected(const om_model* m, const double* theta, double* mu_out) {
    return evaluate(m, theta, 0, mu_out, NULL, NULL);
}

int om_nll(const om_model* m, const double* theta, double* nll, double* grad) {
    return evaluate(m, theta, grad != NULL, NULL, nll, grad);
}

/* a1 values only: Q, mu, sigma, Phi(mu/sigma) on the grid */
int om_quench(const om_model* m, const double* theta, double* Q, double* mu, double* sig, double* den) {
    int st = check_model(m); if (st) return st;
    NP = 0;
    int N = m->n_grid, K = m->K;
    dual th[OPMAX];
    for (int j = 0; j < K + 7; ++j) th[j] = dc(theta[j]);
    work w; memset(&w, 0, sizeof w);
    w.Q = calloc(N, sizeof(dual)); w.mu = calloc(N, sizeof(dual)); w.sig = calloc(N, sizeof(dual)); w.den = calloc(N, sizeof(dual));
    st = stage_a1(m, th, &w, 1.0, 1.0);   /* the map of unit Birks multiplier */
    for (int i = 0; i < N; ++i) {
        if (Q) Q[i] = w.Q[i].v;
        if (mu) mu[i] = w.mu[i].v;
        if (sig) sig[i] = w.sig[i].v;
        if (den) den[i] = w.den[i].v;
    }
    work_free(&w);
    return st;
}

/* a2 + a3 values: the response matrix R [m_hi][n_grid] of the first set of species (may be
 * NULL) and the species spectra v [m_hi][K] (may be NULL). */
int om_response(const om_model* m, const double* theta, double* R, double* v) {
    int st = check_model(m); if (st) return st;
    NP = 0;
    int N = m->n_grid, K = m->K, M = m->m_hi;
    dual th[OPMAX];
    for (int j = 0; j < K + 7; ++j) th[j] = dc(theta[j]);
    work w;
    w.Q = calloc(N, sizeof(dual)); w.mu = calloc(N, sizeof(dual)); w.sig = calloc(N, sizeof(dual));
    w.den = calloc(N, sizeof(dual)); w.v = calloc((size_t)M * K, sizeof(dual));
    double xi[OM_MAX_SETS];
    int set_of[OPMAX];
    const int nset = quench_sets(m, xi, set_of);
    for (int c = 0; c < nset && !st; ++c) {   /* R of the first set */
        st = stage_a1(m, th, &w, xi[c], 1.0);
        if (!st) stage_a23(m, &w, c == 0 ? R : NULL, NULL, NULL, set_of, c, -1);
    }
    if (!st && v) for (size_t j = 0; j < (size_t)M * K; ++j) v[j] = w.v[j].v;
    work_free(&w);
    return st;
}

/* a5 alone on a plain vector x[0..m_hi): y[m_hi - m_lo] */
int om_pileup(const om_model* m, double eps, const double* x, double* y) {
    NP = 0;
    int M = m->m_hi, nw = m->m_hi - m->m_lo;
    dual* xd = calloc(M, sizeof(dual)); dual* yd = calloc(nw, sizeof(dual));
    for (int r = 0; r < M; ++r) xd[r] = dc(x[r]);
    pileup_window(m, dc(eps), xd, 1, yd);
    for (int j = 0; j < nw; ++j) y[j] = yd[j].v;
    free(xd); free(yd);
    return OM_OK;
}

/* radial bin probabilities of one class at s_r, and d/ds_r */
int om_radial(const om_model* m, double s_r, int cls, double* p, double* dp) {
    NP = 1;
    dual* pd = calloc(m->n_rad, sizeof(dual));
    radial_probs(m, dvar(s_r, 0), cls, pd);
    for (int b = 0; b < m->n_rad; ++b) { p[b] = pd[b].v; if (dp) dp[b] = pd[b].d[0]; }
    free(pd);
    NP = 0;
    return OM_OK;
}

/* a6 alone: sum_j [mu_j - n_j + n_j ln(n_j/mu_j)] with Neumaier compensation */
int om_poisson_nll(int n, const double* counts, const double* mu, double* out) {
    NP = 0;
    nsum acc; acc.s = dc(0.0); acc.c = dc(0.0);
    for (int j = 0; j < n; ++j) {
        dual t;
        if (bin_term(counts[j], dc(mu[j]), &t)) { *out = INFINITY; return OM_EDOMAIN; }
        nsum_add(&acc, &t);
    }
    *out = acc.s.v + acc.c.v;
    return OM_OK;
}

/* ---------------------------------------------------------------- fit (minimiser) */

static int cholesky_solve(int n, double* A, const double* b, double* x) {
    /* A (n x n, row-major) overwritten by its Cholesky factor; solves A x = b */
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return -1;
        A[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / A[j * n + j];
        }
    }
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= A[i * n + k] * x[k];
        x[i] = t / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = x[i];
        for (int k = i + 1; k < n; ++k) t -= A[k * n + i] * x[k];
        x[i] = t / A[i * n + i];
    }
    return 0;
}

/* Damped Newton fit.  info[0] = -lnL, info[1] = EDM, info[2] = iterations, info[3] = status.
 * cov (P x P, may be NULL): inverse Hessian on the free set at the optimum (0 elsewhere). */
/* -lnL (and gradient) of the objective a fit minimises: one model, or the several energy
 * estimators of one dataset (om_nll_est). */
typedef int (*om_objective)(const void* ctx, const double* theta, double* f, double* g);

typedef struct { const om_model* m; int E; } est_ctx;

static int obj_single(const void* ctx, const double* theta, double* f, double* g) {
    return om_nll((const om_model*)ctx, theta, f, g);
}

static int fit_core(om_objective om_obj, const void* ctx, int P, const double* theta0, const unsigned char* free_mask,
                    const double* lo, const double* hi, double tol_edm, int max_iter,
                    double* theta_out, double* info, double* cov);

int om_fit(const om_model* m, const double* theta0, const unsigned char* free_mask,
           const double* lo, const double* hi, double tol_edm, int max_iter,
           double* theta_out, double* info, double* cov) {
    return fit_core(obj_single, m, m->K + 7, theta0, free_mask, lo, hi, tol_edm, max_iter, theta_out, info, cov);
}

/* Several energy estimators of one dataset (Sec. 3: the charge, the number of detected
 * photons and the number of fired channels, each an observable N_x with its own response
 * R_x of Eq. 1), fitted jointly.  Reading: the estimators see the same events, so the
 * deposited-energy spectra and everything that acts on them before the detector response
 * are shared -- the rates, the Birks constant kB, the pile-up probability eps and the radial
 * scale s_r -- while each estimator has its own response parameters (LY, a, b, c), binning,
 * window, random-trigger spectrum and data; -lnL is the sum of the estimators' -lnL (their
 * histograms enter as separate terms, as the several terms of Eq. 4 do).  The radial and
 * pulse-shape terms belong to estimator 0 only.  Joint parameter vector (P = K + 7 + 4 (E - 1)):
 *   [r_0 .. r_{K-1}, LY_0, a_0, b_0, c_0, kB, eps, s_r, LY_1, a_1, b_1, c_1, ..., c_{E-1}]
 * so that E = 1 is the single model.  Estimator e is evaluated at
 *   [r_0 .. r_{K-1}, LY_e, a_e, b_e, c_e, kB, eps, s_r]. */
int om_est_theta(int K, int e, const double* theta, double* th_e) {
    for (int k = 0; k < K; ++k) th_e[k] = theta[k];
    const int src = e == 0 ? K : K + 7 + 4 * (e - 1);
    for (int j = 0; j < 4; ++j) th_e[K + j] = theta[src + j];
    for (int j = 4; j < 7; ++j) th_e[K + j] = theta[K + j];
    return OM_OK;
}

int om_nll_est(const om_model* ms, int E, const double* theta, double* nll, double* grad) {
    if (E < 1) return OM_EINVAL;
    const int K = ms[0].K, P = K + 7 + 4 * (E - 1);
    if (P > OPMAX) return OM_EINVAL;
    for (int e = 1; e < E; ++e)
        if (ms[e].K != K || ms[e].n_rad > 0 || ms[e].n_psd > 0 || ms[e].n_r2 + ms[e].n_p2 > 0) return OM_EINVAL;
    double f = 0.0, fe, th[OPMAX], ge[OPMAX];
    if (grad) memset(grad, 0, (size_t)P * sizeof(double));
    int st = OM_OK;
    for (int e = 0; e < E; ++e) {
        om_est_theta(K, e, theta, th);
        const int s = om_nll(&ms[e], th, &fe, grad ? ge : NULL);
        if (s && s != OM_EDOMAIN) return s;
        if (s) st = s;
        f += fe;
        if (grad) {
            const int src = e == 0 ? K : K + 7 + 4 * (e - 1);
            for (int k = 0; k < K; ++k) grad[k] += ge[k];
            for (int j = 0; j < 4; ++j) grad[src + j] += ge[K + j];
            for (int j = 4; j < 7; ++j) grad[K + j] += ge[K + j];
        }
    }
    *nll = f;
    return st;
}

static int obj_est(const void* ctx, const double* theta, double* f, double* g) {
    const est_ctx* c = (const est_ctx*)ctx;
    return om_nll_est(c->m, c->E, theta, f, g);
}

int om_fit_est(const om_model* ms, int E, const double* theta0, const unsigned char* free_mask,
               const double* lo, const double* hi, double tol_edm, int max_iter,
               double* theta_out, double* info, double* cov) {
    if (E < 1 || ms[0].K + 7 + 4 * (E - 1) > OPMAX) return OM_EINVAL;
    est_ctx c = {ms, E};
    return fit_core(obj_est, &c, ms[0].K + 7 + 4 * (E - 1), theta0, free_mask, lo, hi, tol_edm, max_iter,
                    theta_out, info, cov);
}

static int fit_core(om_objective om_obj, const void* ctx, int P, const double* theta0, const unsigned char* free_mask,
                    const double* lo, const double* hi, double tol_edm, int max_iter,
                    double* theta_out, double* info, double* cov) {
    int st = OM_ENOTCONV, it;
    double th[OPMAX], g[OPMAX], gp[OPMAX], gm[OPMAX], tp[OPMAX], H[OPMAX * OPMAX], Hc[OPMAX * OPMAX];
    double step[OPMAX], rhs[OPMAX], f = 0, edm = INFINITY;
    int idx[OPMAX], nf = 0;
    memcpy(th, theta0, P * sizeof(double));
    for (int j = 0; j < P; ++j) th[j] = fmin(fmax(th[j], lo[j]), hi[j]);
    for (it = 0; it < max_iter; ++it) {
        int e = om_obj(ctx, th, &f, g);
        if (e) { st = e; break; }
        nf = 0;
        for (int j = 0; j < P; ++j) {
            if (!free_mask[j]) continue;
            if (th[j] <= lo[j] && g[j] > 0) continue;   /* pinned at the lower bound */
            if (th[j] >= hi[j] && g[j] < 0) continue;   /* pinned at the upper bound */
            idx[nf++] = j;
        }
        /* central-difference Hessian of the exact gradient on the free set */
        for (int a = 0; a < nf; ++a) {
            int j = idx[a];
            double h = 1e-4 * fmax(fabs(th[j]), 1e-3);
            double up = th[j] + h, dn = th[j] - h;
            if (dn < lo[j]) dn = th[j];
            if (up > hi[j]) up = th[j];
            if (up == dn) return OM_EINVAL;
            memcpy(tp, th, P * sizeof(double)); tp[j] = up;
            double fd;
            if ((e = om_obj(ctx, tp, &fd, gp))) return e;
            memcpy(tp, th, P * sizeof(double)); tp[j] = dn;
            if (dn == th[j]) memcpy(gm, g, P * sizeof(double));
            else if ((e = om_obj(ctx, tp, &fd, gm))) return e;
            for (int b = 0; b < nf; ++b) H[b * nf + a] = (gp[idx[b]] - gm[idx[b]]) / (up - dn);
        }
        for (int a = 0; a < nf; ++a)
            for (int b = 0; b < a; ++b) { double s = 0.5 * (H[a * nf + b] + H[b * nf + a]); H[a * nf + b] = H[b * nf + a] = s; }
        for (int a = 0; a < nf; ++a) rhs[a] = -g[idx[a]];
        double damp = 0.0;
        for (;;) {
            memcpy(Hc, H, (size_t)nf * nf * sizeof(double));
            for (int a = 0; a < nf; ++a) Hc[a * nf + a] += damp * fabs(H[a * nf + a]);
            if (cholesky_solve(nf, Hc, rhs, step) == 0) break;
            damp = damp == 0.0 ? 1e-8 : damp * 10.0;
            if (damp > 1e6) return OM_ENOTCONV;
        }
        edm = 0.0;
        for (int a = 0; a < nf; ++a) edm -= 0.5 * g[idx[a]] * step[a];
        if (cov && damp == 0.0) {
            memset(cov, 0, (size_t)P * P * sizeof(double));
            for (int a = 0; a < nf; ++a) {
                double ea[OPMAX], col[OPMAX];
                for (int b = 0; b < nf; ++b) ea[b] = (a == b);
                memcpy(Hc, H, (size_t)nf * nf * sizeof(double));
                cholesky_solve(nf, Hc, ea, col);
                for (int b = 0; b < nf; ++b) cov[idx[b] * P + idx[a]] = col[b];
            }
        }
        if (edm < tol_edm && damp == 0.0) { st = OM_OK; break; }
        /* backtracking line search on the projected step */
        double alpha = 1.0, slope = 0.0, fn = 0.0;
        for (int a = 0; a < nf; ++a) slope += g[idx[a]] * step[a];
        int ok = 0;
        for (int ls = 0; ls < 50; ++ls) {
            memcpy(tp, th, P * sizeof(double));
            for (int a = 0; a < nf; ++a) { int j = idx[a]; tp[j] = fmin(fmax(th[j] + alpha * step[a], lo[j]), hi[j]); }
            e = om_obj(ctx, tp, &fn, NULL);
            if (!e && fn <= f + 1e-4 * alpha * slope) { ok = 1; break; }
            alpha *= 0.5;
        }
        if (!ok) { st = OM_ENOTCONV; break; }
        memcpy(th, tp, P * sizeof(double));
    }
    memcpy(theta_out, th, P * sizeof(double));
    if (info) { info[0] = f; info[1] = edm; info[2] = it; info[3] = st; }
    return st;
}
